"""GPU evaluation of the same seeded input recipe as rf_inputs (inputs only,
no method arithmetic): K-mode Fourier fields -> metric factor L and drift
w for a batch of images, evaluated with torch outer products on the device.
Used to generate the warm-start network's training data at scale."""
from __future__ import annotations

import math

import numpy as np
import torch

from . import FIELD_A, FIELD_B, FIELD_PHI, FIELD_THETA, rng_for


def _field(n, h, K, rng, device):
    kmax = int(math.ceil(math.sqrt(K))) + 1
    ks = []
    while len(ks) < K:
        k = rng.integers(-kmax, kmax + 1, size=2)
        if k[0] != 0 or k[1] != 0:
            ks.append(k)
    ks = np.array(ks, dtype=np.float64)
    c = rng.standard_normal(K) / np.linalg.norm(ks, axis=1)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=K)
    x = torch.arange(n, dtype=torch.float64, device=device) * h
    ax = 2 * math.pi * torch.as_tensor(ks[:, 0], device=device)[:, None] * x[None, :] + \
        torch.as_tensor(phi, device=device)[:, None]
    ay = 2 * math.pi * torch.as_tensor(ks[:, 1], device=device)[:, None] * x[None, :]
    cc = torch.as_tensor(c, device=device)[:, None, None]
    f = (cc * (torch.cos(ay)[:, :, None] * torch.cos(ax)[:, None, :] -
               torch.sin(ay)[:, :, None] * torch.sin(ax)[:, None, :])).sum(0)
    lo, hi = f.min(), f.max()
    return (f - lo) / (hi - lo)


def randers_fields_batch(seeds, n, h, K, eps=1e-6, omega_scale=0.3, device="cuda"):
    """float32 [len(seeds), 5, n, n] raw fields (L11, L21, L22, wx, wy) on
    `device`, one image per seed, |w|_2 = omega_scale."""
    out = torch.empty((len(seeds), 5, n, n), dtype=torch.float32, device=device)
    for b, seed in enumerate(seeds):
        th = math.pi * _field(n, h, K, rng_for(seed, FIELD_THETA), device)
        a = 0.5 * 4.0 ** _field(n, h, K, rng_for(seed, FIELD_A), device)
        bb = 0.5 * 4.0 ** _field(n, h, K, rng_for(seed, FIELD_B), device)
        ct, st = torch.cos(th), torch.sin(th)
        m11 = a * a * ct * ct + bb * bb * st * st
        m12 = (a * a - bb * bb) * ct * st
        m22 = a * a * st * st + bb * bb * ct * ct
        l11 = torch.sqrt(m11 - eps)
        l21 = m12 / l11
        l22 = torch.sqrt(m22 - eps - l21 * l21)
        ph = 2 * math.pi * _field(n, h, K, rng_for(seed, FIELD_PHI), device)
        out[b, 0], out[b, 1], out[b, 2] = l11, l21, l22
        out[b, 3], out[b, 4] = omega_scale * torch.cos(ph), omega_scale * torch.sin(ph)
    return out


def random_sources_batch(seeds, n, lo=1, hi=8, device="cuda"):
    """uint8 [len(seeds), n, n] masks with lo..hi random source nodes each,
    and the list of (image, row, column) sources."""
    src = torch.zeros((len(seeds), n, n), dtype=torch.uint8, device=device)
    pts = []
    for b, seed in enumerate(seeds):
        rng = rng_for(seed, 101)
        k = int(rng.integers(lo, hi + 1))
        idx = rng.choice(n * n, size=k, replace=False)
        for p in idx:
            pts.append((b, int(p) // n, int(p) % n))
            src[b, int(p) // n, int(p) % n] = 1
    return src, pts
