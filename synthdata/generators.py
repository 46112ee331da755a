"""Seeded image / mask / workload generators (no method arithmetic here).

Recipe for one channel (numpy PCG64 stream per channel):
  * start from the constant 96;
  * add 20 anisotropic Gaussians: centre uniform in [0,W)x[0,H), the two
    standard deviations log-uniform in [0.02, 0.25]*min(W,H), orientation
    uniform in [0, pi), amplitude uniform in [-100, 160];
  * paint 8 axis-aligned rectangles (later ones overwrite earlier ones):
    width/height uniform in [0.05, 0.3]*(W, H), top-left uniform so that the
    rectangle fits, value uniform in [0, 255];
  * add N(0, 2) noise and clip to [0, 255].
Masks: exactly round(d*N) distinct pixels drawn with Generator.choice from
their own stream.
"""

from __future__ import annotations

import math

import numpy as np

N_GAUSS = 20
N_RECT = 8


def synth_image(height: int, width: int, seed: int, dtype=np.float64) -> np.ndarray:
    """One grey channel of shape (height, width) on the [0, 255] scale."""
    rng = np.random.Generator(np.random.PCG64(seed))
    H, W = int(height), int(width)
    img = np.full((H, W), 96.0, dtype=np.float64)
    ys = np.arange(H, dtype=np.float64)[:, None]
    xs = np.arange(W, dtype=np.float64)[None, :]
    smin = float(min(W, H))
    for _ in range(N_GAUSS):
        cx = rng.uniform(0.0, W)
        cy = rng.uniform(0.0, H)
        s1 = math.exp(rng.uniform(math.log(0.02 * smin), math.log(0.25 * smin)))
        s2 = math.exp(rng.uniform(math.log(0.02 * smin), math.log(0.25 * smin)))
        ang = rng.uniform(0.0, math.pi)
        amp = rng.uniform(-100.0, 160.0)
        ca, sa = math.cos(ang), math.sin(ang)
        # separable evaluation of the rotated quadratic form, row by row blocks
        dx = xs - cx
        for y0 in range(0, H, 512):
            dy = ys[y0:y0 + 512] - cy
            a = dx * ca + dy * sa
            b = -dx * sa + dy * ca
            img[y0:y0 + 512] += amp * np.exp(-0.5 * ((a / s1) ** 2 + (b / s2) ** 2))
    for _ in range(N_RECT):
        rw = max(1, int(round(rng.uniform(0.05, 0.3) * W)))
        rh = max(1, int(round(rng.uniform(0.05, 0.3) * H)))
        x0 = int(rng.integers(0, W - rw + 1))
        y0 = int(rng.integers(0, H - rh + 1))
        img[y0:y0 + rh, x0:x0 + rw] = rng.uniform(0.0, 255.0)
    img += rng.normal(0.0, 2.0, size=(H, W))
    np.clip(img, 0.0, 255.0, out=img)
    return img.astype(dtype)


def synth_rgb(height: int, width: int, seeds=(1, 2, 3), dtype=np.float32) -> np.ndarray:
    """Planar (channels, H, W) image, one independent stream per channel."""
    return np.stack([synth_image(height, width, s, dtype) for s in seeds])


def random_mask(height: int, width: int, density: float, seed: int) -> np.ndarray:
    """uint8 (H, W) mask with exactly round(density*H*W) ones (at least one)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = height * width
    m = int(round(density * n))
    m = min(max(m, 1), n)
    idx = rng.choice(n, size=m, replace=False)
    c = np.zeros(n, dtype=np.uint8)
    c[idx] = 1
    return c.reshape(height, width)


BATCH_SIZES = ((256, 256), (512, 384), (1024, 768), (1920, 1080), (2048, 1080))


def batch_specs(count: int = 64, seed: int = 200):
    """Uneven batch: list of dicts (width, height, channels, density, seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        w, h = BATCH_SIZES[int(rng.integers(0, len(BATCH_SIZES)))]
        ch = 3 if rng.uniform() < 0.5 else 1
        d = float(rng.uniform(0.01, 0.10))
        out.append(dict(width=w, height=h, channels=ch, density=d, seed=seed + 1 + i))
    return out


def serving_stream(count: int = 2000, rate: float = 200.0, seed: int = 400):
    """Poisson arrivals; area log-uniform in [512^2, 3840*2160], aspect 16:9,
    sides rounded to multiples of 8; grey/RGB with p=1/2; 70/25/5 mix of
    inpaint / tonal / densify-to-3%."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    lo, hi = math.log(512.0 * 512.0), math.log(3840.0 * 2160.0)
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        area = math.exp(rng.uniform(lo, hi))
        w = max(8, int(round(math.sqrt(area * 16.0 / 9.0) / 8.0)) * 8)
        h = max(8, int(round(math.sqrt(area * 9.0 / 16.0) / 8.0)) * 8)
        w, h = min(w, 3840), min(h, 2160)
        ch = 3 if rng.uniform() < 0.5 else 1
        r = rng.uniform()
        kind = "inpaint" if r < 0.70 else ("tonal" if r < 0.95 else "densify")
        d = float(rng.uniform(0.01, 0.10))
        out.append(dict(id=i, arrival=t, width=w, height=h, channels=ch, kind=kind,
                        density=d, seed=seed + 1 + i))
    return out


def serving_inputs(spec: dict, base: np.ndarray):
    """Image and mask of one serving request: a crop of a shared synthetic
    RGB base image (at least the request's size) at an offset drawn from the
    request's seed, channel 0 only for grey requests, and a Bernoulli mask
    of the request's density (fast to draw for thousands of requests)."""
    rng = np.random.Generator(np.random.PCG64(spec["seed"]))
    H, W = spec["height"], spec["width"]
    y0 = int(rng.integers(0, base.shape[1] - H + 1))
    x0 = int(rng.integers(0, base.shape[2] - W + 1))
    f = base[: spec["channels"], y0:y0 + H, x0:x0 + W]
    f = np.ascontiguousarray(f, dtype=np.float32)
    m = (rng.random((H, W)) < spec["density"]).astype(np.uint8)
    if not m.any():
        m[H // 2, W // 2] = 1
    return f, m
