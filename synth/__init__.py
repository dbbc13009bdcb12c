"""Seeded synthetic workloads for the Köhler contrast-curve path.

The paper's own inputs (the 18-Mpixel "Tulips" photograph, "Lenna" and a
YFCC100M car video, Section 4) are not available, so these generators stand in
for them with the same sizes, value ranges and spatial structure.  The same
bytes feed the CPU oracle and the CUDA library; this module holds none of the
method's arithmetic (no pair, boundary, histogram or contrast computation).

Every generator draws from ``numpy.random.Generator(PCG64(seed))``; continuous
values are rounded half-to-even (``np.rint``) and clipped to the value range.

Workloads (base seeds in ``SEEDS``):
  blobs_256            256 x 256 uint8, linear gradient + 6 Gaussian blobs + uniform noise in [-8, 8]
  voronoi_18mp         5184 x 3456 uint8, 200-seed Voronoi regions, levels from a 3-component
                       Gaussian mixture (means 50/120/200, sd 15), Gaussian noise sd 4
  voronoi_batch96      96 uint8 Voronoi images, sizes uniform over 5 resolutions, 20-400 seeds,
                       noise sd 2-10
  cosine_u16_batch16   16 x 2048 x 2048 uint16 (12-bit), sum of 32 random 2-D cosines mapped to
                       [0, 4095], Gaussian noise sd 20
  video_stream         uint8 frames at mixed resolutions (60 % 1920x1080, 25 % 3840x2160,
                       15 % 640x480): 10 moving ellipses on a drifting gradient, noise sd 5,
                       Poisson arrivals at 240 frames/s
"""
from __future__ import annotations

import numpy as np

SEEDS = {
    "blobs_256": 1001,
    "voronoi_18mp": 2002,
    "voronoi_batch96": 3003,
    "cosine_u16_batch16": 4004,
    "video_stream": 5005,
}

BATCH96_SIZES = ((320, 240), (640, 480), (1280, 720), (1920, 1080), (4096, 3072))
VIDEO_SIZES = ((1920, 1080), (3840, 2160), (640, 480))
VIDEO_PROBS = (0.60, 0.25, 0.15)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _to_dtype(x: np.ndarray, hi: int, dtype) -> np.ndarray:
    return np.clip(np.rint(x), 0, hi).astype(dtype)


# ---------------------------------------------------------------- small / test images
def random_image(seed: int, w: int, h: int, M: int, dtype=np.uint8) -> np.ndarray:
    """Independent uniform values in [0, M[ (worst case for locality)."""
    return rng(seed).integers(0, M, size=(h, w), dtype=np.int64).astype(dtype)


def smooth_image(seed: int, w: int, h: int, M: int, dtype=np.uint8, noise_sd: float = 3.0) -> np.ndarray:
    """Random piecewise-smooth field: a few Gaussian bumps on a gradient plus noise,
    spanning most of [0, M[.  Used for ragged-shape parity cases."""
    g = rng(seed)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    f = g.uniform(0.2, 0.8) * M + g.uniform(-0.2, 0.2) * M * (xx / max(w, 1) - 0.5)
    for _ in range(4):
        cx, cy = g.uniform(0, w), g.uniform(0, h)
        s = g.uniform(0.1, 0.4) * max(w, h) + 1.0
        f += g.uniform(-0.35, 0.35) * M * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * s * s))
    f += g.normal(0.0, noise_sd * M / 256.0, size=(h, w))
    return _to_dtype(f, M - 1, dtype)


# ---------------------------------------------------------------- 256 x 256 blobs
def blobs_image(seed: int = SEEDS["blobs_256"], w: int = 256, h: int = 256) -> np.ndarray:
    g = rng(seed)
    yy, xx = np.mgrid[0:h, 0:w].astype(np.float64)
    ang = g.uniform(0, 2 * np.pi)
    lo, hi = g.uniform(20, 80), g.uniform(150, 220)
    proj = (xx - w / 2) * np.cos(ang) + (yy - h / 2) * np.sin(ang)
    proj = (proj - proj.min()) / max(proj.max() - proj.min(), 1e-9)
    f = lo + (hi - lo) * proj
    for _ in range(6):
        cx, cy = g.uniform(0, w), g.uniform(0, h)
        s = g.uniform(8, 40)
        amp = g.uniform(-120, 120)
        f += amp * np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * s * s))
    f += g.integers(-8, 9, size=(h, w))
    return _to_dtype(f, 255, np.uint8)


# ---------------------------------------------------------------- Voronoi images
def voronoi_labels(g: np.random.Generator, w: int, h: int, n_seeds: int) -> np.ndarray:
    """Index of the nearest of n_seeds uniform random seeds for every pixel centre."""
    from scipy.spatial import cKDTree

    seeds = np.stack([g.uniform(0, w, n_seeds), g.uniform(0, h, n_seeds)], axis=1)
    tree = cKDTree(seeds)
    labels = np.empty((h, w), np.int32)
    xs = np.arange(w, dtype=np.float64) + 0.5
    rows = max(1, (1 << 21) // w)
    for y0 in range(0, h, rows):
        y1 = min(h, y0 + rows)
        yy = np.repeat(np.arange(y0, y1, dtype=np.float64) + 0.5, w)
        pts = np.stack([np.tile(xs, y1 - y0), yy], axis=1)
        _, idx = tree.query(pts, k=1, workers=-1)
        labels[y0:y1] = idx.reshape(y1 - y0, w)
    return labels


def voronoi_levels(g: np.random.Generator, n: int) -> np.ndarray:
    """Region levels from an equal-weight 3-component Gaussian mixture (50/120/200, sd 15)."""
    comp = g.integers(0, 3, size=n)
    return np.array([50.0, 120.0, 200.0])[comp] + g.normal(0.0, 15.0, size=n)


def voronoi_image(seed: int, w: int, h: int, n_seeds: int, noise_sd: float, labels=None) -> np.ndarray:
    g = rng(seed)
    if labels is None:
        labels = voronoi_labels(g, w, h, n_seeds)
        n = n_seeds
    else:
        n = int(labels.max()) + 1
    lv = voronoi_levels(g, n)
    f = lv[labels] + g.normal(0.0, noise_sd, size=(h, w))
    return _to_dtype(f, 255, np.uint8)


def voronoi_18mp(seed: int = SEEDS["voronoi_18mp"]) -> np.ndarray:
    """One 5184 x 3456 Voronoi image (200 seeds, noise sd 4)."""
    return voronoi_image(seed, 5184, 3456, 200, 4.0)


def voronoi_18mp_pool(n: int, seed: int = SEEDS["voronoi_18mp"]) -> list:
    """n distinct 5184 x 3456 images: image 0 is ``voronoi_18mp(seed)``; the others
    share its region map but draw their own region levels and noise (seed + i)."""
    g = rng(seed)
    labels = voronoi_labels(g, 5184, 3456, 200)
    out = [voronoi_18mp(seed)]
    for i in range(1, n):
        out.append(voronoi_image(seed + i, 5184, 3456, 200, 4.0, labels=labels))
    return out


def batch96_specs(seed: int = SEEDS["voronoi_batch96"], n: int = 96):
    """Per-image (w, h, n_seeds, noise_sd, image_seed) of the 96-image batch."""
    g = rng(seed)
    out = []
    for i in range(n):
        w, h = BATCH96_SIZES[int(g.integers(0, len(BATCH96_SIZES)))]
        ns = int(g.integers(20, 401))
        sd = float(g.uniform(2.0, 10.0))
        out.append((w, h, ns, sd, seed + 1 + i))
    return out


def _voronoi_spec(spec):
    w, h, ns, sd, s = spec
    return voronoi_image(s, w, h, ns, sd)


def voronoi_batch(specs, workers: int = 1) -> list:
    """Images of `specs` (see batch96_specs); workers > 1 renders them in a pool
    of spawned processes (safe after CUDA is initialised), same bytes."""
    if workers <= 1 or len(specs) < 2:
        return [_voronoi_spec(sp) for sp in specs]
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor

    with ProcessPoolExecutor(max_workers=min(workers, len(specs)), mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_voronoi_spec, specs))


# ---------------------------------------------------------------- 12-bit cosine fields
def cosine_u16(seed: int, w: int = 2048, h: int = 2048, n_waves: int = 32, noise_sd: float = 20.0) -> np.ndarray:
    """Sum of n_waves 2-D cosines with integer frequencies of at most 8 cycles per
    image, mapped affinely to [0, 4095], plus Gaussian noise; 12-bit values in uint16."""
    g = rng(seed)
    u = g.integers(-8, 9, size=n_waves).astype(np.float64)
    v = g.integers(-8, 9, size=n_waves).astype(np.float64)
    ph = g.uniform(0, 2 * np.pi, size=n_waves)
    amp = g.uniform(0.0, 1.0, size=n_waves)
    ax = 2 * np.pi * np.outer(u, np.arange(w) / w) + ph[:, None]      # (n, w)
    ay = 2 * np.pi * np.outer(v, np.arange(h) / h)                    # (n, h)
    # cos(ax + ay) = cos ax cos ay - sin ax sin ay, summed over waves
    f = (amp[:, None] * np.cos(ay)).T @ np.cos(ax) - (amp[:, None] * np.sin(ay)).T @ np.sin(ax)
    f = (f - f.min()) / max(f.max() - f.min(), 1e-12) * 4095.0
    f += g.normal(0.0, noise_sd, size=(h, w))
    return _to_dtype(f, 4095, np.uint16)


def cosine_u16_batch(n: int = 16, seed: int = SEEDS["cosine_u16_batch16"], w: int = 2048, h: int = 2048) -> list:
    return [cosine_u16(seed + i, w, h) for i in range(n)]


# ---------------------------------------------------------------- video stream
class VideoScene:
    """Ten ellipses moving at constant velocity over a slowly drifting gradient.
    State is in normalised coordinates, so every resolution renders the same scene."""

    def __init__(self, seed: int = SEEDS["video_stream"], n_ellipses: int = 10):
        g = rng(seed)
        self.c = g.uniform(0.1, 0.9, size=(n_ellipses, 2))
        self.v = g.uniform(-0.004, 0.004, size=(n_ellipses, 2))
        self.ax = g.uniform(0.03, 0.15, size=(n_ellipses, 2))
        self.theta = g.uniform(0, np.pi, size=n_ellipses)
        self.level = g.uniform(0, 255, size=n_ellipses)
        self.bg0 = g.uniform(60, 120)
        self.bg_amp = g.uniform(20, 60)
        self.bg_rate = g.uniform(0.002, 0.01)
        self.seed = seed

    def frame(self, k: int, w: int, h: int, noise_sd: float = 5.0) -> np.ndarray:
        g = rng(self.seed * 7919 + 1 + k)
        xn = (np.arange(w, dtype=np.float32) / np.float32(w))[None, :]
        yn = (np.arange(h, dtype=np.float32) / np.float32(h))[:, None]
        a = self.bg_rate * k
        f = self.bg0 + self.bg_amp * (np.cos(a) * xn + np.sin(a) * yn)
        for i in range(len(self.level)):
            cx, cy = (self.c[i] + k * self.v[i]) % 1.0
            ct, st = np.cos(self.theta[i]), np.sin(self.theta[i])
            # only pixels within the larger semi-axis of the centre can be inside
            rx = self.ax[i].max()
            x_a, x_b = max(0, int(np.floor((cx - rx) * w)) - 1), min(w, int(np.ceil((cx + rx) * w)) + 2)
            y_a = max(0, int(np.floor((cy - rx * w / h) * h)) - 1)
            y_b = min(h, int(np.ceil((cy + rx * w / h) * h)) + 2)
            if x_a >= x_b or y_a >= y_b:
                continue
            dx, dy = xn[:, x_a:x_b] - cx, (yn[y_a:y_b] - cy) * (h / w)
            u = (dx * ct + dy * st) / self.ax[i, 0]
            v = (-dx * st + dy * ct) / self.ax[i, 1]
            sub = f[y_a:y_b, x_a:x_b]
            f[y_a:y_b, x_a:x_b] = np.where(u * u + v * v <= 1.0, np.float32(self.level[i]), sub)
        f = f + g.normal(0.0, noise_sd, size=(h, w)).astype(np.float32)
        return _to_dtype(f, 255, np.uint8)


def video_schedule(n_frames: int = 2000, fps: float = 240.0, seed: int = SEEDS["video_stream"]):
    """(arrival times in seconds, resolution index per frame) of the served stream:
    exponential inter-arrival times at the given rate, resolutions drawn with
    probabilities 60/25/15 % over 1920x1080, 3840x2160, 640x480."""
    g = rng(seed + 17)
    arrivals = np.cumsum(g.exponential(1.0 / fps, size=n_frames))
    res = g.choice(len(VIDEO_SIZES), size=n_frames, p=np.array(VIDEO_PROBS))
    return arrivals, res
