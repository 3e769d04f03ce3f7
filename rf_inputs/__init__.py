"""Seeded synthetic inputs for the Randers eikonal solver.

This module is the one piece that both the FP64 oracle tests and the CUDA
path consume.  It generates *inputs only* -- smooth random Fourier fields,
metric factors, drift fields, source masks and loss gradients -- and holds
none of the method's arithmetic (no projection, no local update, no sweep,
no adjoint).

Recipe (stand-in for the paper's synthetic and wildfire workloads; the
Sim2Real-Fire data is not used):

* a K-mode field f(x) = sum_m c_m cos(2 pi k_m . x + phi_m) on physical
  coordinates x = (j h, i h); k_m integer vectors uniform in
  [-kmax, kmax]^2 minus the origin with kmax = ceil(sqrt(K)) + 1;
  c_m ~ N(0,1)/|k_m|; phi_m ~ U[0, 2 pi); min-max normalised to [0, 1];
* theta = pi f_theta, a = 0.5 * 4**f_a, b = 0.5 * 4**f_b (so a, b in
  [0.5, 2] and the speed anisotropy is at most 4);
  M = R(theta) diag(a^2, b^2) R(theta)^T, and the raw factor L is the
  Cholesky factor of M - eps I (the solver rebuilds M = L L^T + eps I);
* drift: direction 2 pi f_phi; magnitude either a constant (e.g. 0.3) or
  a smooth field r_max * f_r;
* every array is rounded to float32 once, so the FP64 oracle and the FP32
  kernels read bit-identical inputs.

Random streams are numpy PCG64 generators keyed by (seed, field id).
"""
from __future__ import annotations

import math

import numpy as np

FIELD_THETA, FIELD_A, FIELD_B, FIELD_PHI, FIELD_R = 0, 1, 2, 3, 4


def rng_for(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream)])))


def fourier_field(ny: int, nx: int, h: float, K: int, rng: np.random.Generator) -> np.ndarray:
    """Smooth random field normalised to [0, 1] (float64, shape (ny, nx))."""
    kmax = int(math.ceil(math.sqrt(K))) + 1
    ks = []
    while len(ks) < K:
        k = rng.integers(-kmax, kmax + 1, size=2)
        if k[0] != 0 or k[1] != 0:
            ks.append(k)
    ks = np.array(ks, dtype=np.float64)
    c = rng.standard_normal(K) / np.linalg.norm(ks, axis=1)
    phi = rng.uniform(0.0, 2.0 * math.pi, size=K)
    x = np.arange(nx, dtype=np.float64) * h
    y = np.arange(ny, dtype=np.float64) * h
    f = np.zeros((ny, nx))
    for m in range(K):
        ax = 2.0 * math.pi * ks[m, 0] * x + phi[m]
        ay = 2.0 * math.pi * ks[m, 1] * y
        # cos(ax + ay) = cos ax cos ay - sin ax sin ay  (separable outer products)
        f += c[m] * (np.outer(np.cos(ay), np.cos(ax)) - np.outer(np.sin(ay), np.sin(ax)))
    lo, hi = f.min(), f.max()
    return (f - lo) / (hi - lo) if hi > lo else np.zeros_like(f)


def metric_factor(theta, a, b, eps):
    """Lower Cholesky factor of R(theta) diag(a^2, b^2) R(theta)^T - eps I."""
    ct, st = np.cos(theta), np.sin(theta)
    m11 = a * a * ct * ct + b * b * st * st
    m12 = (a * a - b * b) * ct * st
    m22 = a * a * st * st + b * b * ct * ct
    l11 = np.sqrt(m11 - eps)
    l21 = m12 / l11
    l22 = np.sqrt(m22 - eps - l21 * l21)
    return l11, l21, l22


def randers_fields(ny, nx, h, K, seed, eps=1e-6, omega="unit", omega_scale=0.3, omega_max=1.2):
    """Raw solver inputs, float32 array (5, ny, nx) = (L11, L21, L22, wx, wy).

    omega="unit": |w|_2 = omega_scale everywhere (direction field);
    omega="field": |w|_2 = omega_max * f_r, a smooth field in [0, omega_max].
    """
    th = math.pi * fourier_field(ny, nx, h, K, rng_for(seed, FIELD_THETA))
    a = 0.5 * 4.0 ** fourier_field(ny, nx, h, K, rng_for(seed, FIELD_A))
    b = 0.5 * 4.0 ** fourier_field(ny, nx, h, K, rng_for(seed, FIELD_B))
    l11, l21, l22 = metric_factor(th, a, b, eps)
    ph = 2.0 * math.pi * fourier_field(ny, nx, h, K, rng_for(seed, FIELD_PHI))
    if omega == "unit":
        r = np.full((ny, nx), float(omega_scale))
    elif omega == "field":
        r = omega_max * fourier_field(ny, nx, h, K, rng_for(seed, FIELD_R))
    else:
        raise ValueError(omega)
    out = np.stack([l11, l21, l22, r * np.cos(ph), r * np.sin(ph)]).astype(np.float32)
    return np.ascontiguousarray(out)


def gb_fields(ny, nx, h, K, seed, drift_max=1.5):
    """Raw fields in the paper's own parameterisation, float32 (5, ny, nx) =
    (g11, g12, g22, b1, b2): G = R(theta) diag(a^2, b^2) R(theta)^T with
    a, b in [0.5, 2] as above (eigenvalues in [0.25, 4]), and a drift of
    direction 2 pi f_phi and magnitude drift_max * f_r -- the kind of
    unconstrained output a network produces, for the projection to act on."""
    th = math.pi * fourier_field(ny, nx, h, K, rng_for(seed, FIELD_THETA))
    a = 0.5 * 4.0 ** fourier_field(ny, nx, h, K, rng_for(seed, FIELD_A))
    b = 0.5 * 4.0 ** fourier_field(ny, nx, h, K, rng_for(seed, FIELD_B))
    ct, st = np.cos(th), np.sin(th)
    g11 = a * a * ct * ct + b * b * st * st
    g12 = (a * a - b * b) * ct * st
    g22 = a * a * st * st + b * b * ct * ct
    ph = 2.0 * math.pi * fourier_field(ny, nx, h, K, rng_for(seed, FIELD_PHI))
    r = drift_max * fourier_field(ny, nx, h, K, rng_for(seed, FIELD_R))
    out = np.stack([g11, g12, g22, r * np.cos(ph), r * np.sin(ph)]).astype(np.float32)
    return np.ascontiguousarray(out)


def piecewise_isotropic(n=80, g_left=1.0, g_right=2.0):
    """The paper's isotropic inverse-experiment truth (App. "Inverse Problem
    Experiments"): G = g I on an n x n grid, g = g_left for columns j < n/2
    and g_right for the rest; zero drift.  float32 (5, n, n) in (g11, g12,
    g22, b1, b2)."""
    g = np.where(np.arange(n)[None, :] < n // 2, g_left, g_right) * np.ones((n, 1))
    z = np.zeros((n, n))
    return np.ascontiguousarray(np.stack([g, z, g, z, z]).astype(np.float32))


def constant_gb(n, g=(1.0, 0.0, 1.0), b=(0.0, 0.0)):
    """Constant (g11, g12, g22, b1, b2) on an n x n grid, float32."""
    vals = list(g) + list(b)
    return np.ascontiguousarray(np.stack([np.full((n, n), float(v)) for v in vals]).astype(np.float32))


def covariate_sample(n, seed, slope_gain=0.5, fuel_gain=0.8, drift_max=0.3):
    """One synthetic wildfire-like sample on an n x n grid (h = 1/(n-1)),
    after the paper's synthetic propagation scenarios (App. "Synthetic
    Propagation Scenarios": terrain g = 1 + alpha |grad z|, high-resistance
    patches, uniform drift, combined multiplicatively):
      spatial covariates  z (a 4-mode Fourier terrain, heights up to 0.25)
                          and fuel (1 inside 3-6 random discs, else 0);
      global covariates   wind (cos, sin) x speed in [0, 1] and a
                          temperature in [0, 1];
      true fields         G = g I with g = (1 + slope_gain |grad z|)
                          (1 + fuel_gain fuel), b = drift_max speed
                          (0.5 + 0.5 temperature) (cos, sin), uniform.
    Returns float32 arrays: Y [n, n, 2] (z, fuel), y [3], gb [5, n, n]."""
    h = 1.0 / (n - 1)
    rng = rng_for(seed, 200)
    z = 0.25 * fourier_field(n, n, h, 4, rng_for(seed, 201))
    gy, gx = np.gradient(z, h)
    slope = np.hypot(gx, gy)
    yy, xx = np.mgrid[0:n, 0:n] * h
    fuel = np.zeros((n, n))
    for _ in range(int(rng.integers(3, 7))):
        cx, cy, r = rng.uniform(0.1, 0.9), rng.uniform(0.1, 0.9), rng.uniform(0.05, 0.15)
        fuel[(xx - cx) ** 2 + (yy - cy) ** 2 < r * r] = 1.0
    th, speed, temp = rng.uniform(0, 2 * math.pi), rng.uniform(0, 1), rng.uniform(0, 1)
    g = (1.0 + slope_gain * slope) * (1.0 + fuel_gain * fuel)
    bmag = drift_max * speed * (0.5 + 0.5 * temp)
    gb = np.stack([g, np.zeros_like(g), g, np.full_like(g, bmag * math.cos(th)), np.full_like(g, bmag * math.sin(th))])
    Y = np.stack([z / 0.25, fuel], axis=-1)
    y = np.array([speed * math.cos(th), speed * math.sin(th), temp])
    return dict(Y=Y.astype(np.float32), y=y.astype(np.float32), gb=np.ascontiguousarray(gb.astype(np.float32)),
                h=h)


def constant_fields(ny, nx, M, w, eps=0.0):
    """Constant metric M (2x2 SPD) and drift w, as raw float32 (5, ny, nx)."""
    M = np.asarray(M, dtype=np.float64)
    l11 = math.sqrt(M[0, 0] - eps)
    l21 = M[0, 1] / l11
    l22 = math.sqrt(M[1, 1] - eps - l21 * l21)
    vals = [l11, l21, l22, float(w[0]), float(w[1])]
    return np.ascontiguousarray(
        np.stack([np.full((ny, nx), v) for v in vals]).astype(np.float32))


def point_sources(ny, nx, points):
    src = np.zeros((ny, nx), np.uint8)
    for (i, j) in points:
        src[i, j] = 1
    return src


def random_sources(ny, nx, count, seed, margin=0):
    rng = rng_for(seed, 100)
    idx = rng.choice((ny - 2 * margin) * (nx - 2 * margin), size=count, replace=False)
    pts = [(margin + int(p) // (nx - 2 * margin), margin + int(p) % (nx - 2 * margin)) for p in idx]
    return point_sources(ny, nx, pts)


def block_source(ny, nx, ci, cj, half=1):
    """(2 half + 1)^2 block of source nodes centred at (ci, cj) (the paper's
    3x3 ignition region for half = 1)."""
    src = np.zeros((ny, nx), np.uint8)
    src[max(0, ci - half):ci + half + 1, max(0, cj - half):cj + half + 1] = 1
    return src


def sparse_loss_grad(ny, nx, frac, seed):
    """A seeded dL/dT: standard normal values on a random `frac` of the cells,
    zero elsewhere (float32)."""
    rng = rng_for(seed, 200)
    n = ny * nx
    k = max(1, int(round(frac * n)))
    idx = rng.choice(n, size=k, replace=False)
    g = np.zeros(n, np.float32)
    g[idx] = rng.standard_normal(k).astype(np.float32)
    return g.reshape(ny, nx)


def observation_mask(ny, nx, frac, seed):
    rng = rng_for(seed, 300)
    n = ny * nx
    k = max(1, int(round(frac * n)))
    m = np.zeros(n, np.uint8)
    m[rng.choice(n, size=k, replace=False)] = 1
    return m.reshape(ny, nx)


# ---- the five workloads (sizes and recipes) ---------------------------------

def config1(seed=0):
    """64x64, h = 1/63, K = 8, |w| = 0.3, one source at node (32, 32)."""
    n = 64
    h = 1.0 / 63
    raw = randers_fields(n, n, h, 8, seed, omega="unit", omega_scale=0.3)
    return dict(raw=raw, src=point_sources(n, n, [(32, 32)]), h=h, eps=1e-6, delta=0.05,
                g=sparse_loss_grad(n, n, 0.05, seed))


def config2(seed=0):
    """512x512, h = 1/511, K = 16, 4 random sources, |w|_2 a smooth field in
    [0, 1.2] projected to |w|_{M^-1} <= 0.6 (delta = 0.4), 1% observations."""
    n = 512
    h = 1.0 / 511
    raw = randers_fields(n, n, h, 16, seed, omega="field", omega_max=1.2)
    return dict(raw=raw, src=random_sources(n, n, 4, seed), h=h, eps=1e-6, delta=0.4,
                g=sparse_loss_grad(n, n, 0.01, seed))


def config_inverse(n=2048, seed=0, nsrc=4):
    """n x n (2048 by default), h = 1/(n-1), K = 16 ground-truth field, |w|=0.3
    direction field, `nsrc` random sources, 0.5% observed cells."""
    h = 1.0 / (n - 1)
    raw = randers_fields(n, n, h, 16, seed, omega="unit", omega_scale=0.3)
    return dict(raw=raw, src=random_sources(n, n, nsrc, seed), h=h, eps=1e-6, delta=0.05,
                g=sparse_loss_grad(n, n, 0.005, seed), obs=observation_mask(n, n, 0.005, seed))


def batch_shapes(count=256, seed=0, lo=64, hi=1024):
    """Grid shapes of the batched workload: long side s ~ U{lo..hi}; half
    square (s x s), half 2:1 (s/2 rows x s columns)."""
    rng = rng_for(seed, 400)
    shapes = []
    for b in range(count):
        s = int(rng.integers(lo, hi + 1))
        if b % 2 == 0:
            shapes.append((s, s))
        else:
            shapes.append((max(2, s // 2), s))
    return shapes
