"""Seeded synthetic grey images and obstacle masks.

This module only draws inputs. It holds none of the geodesic arithmetic: the
CUDA library and the CPU oracle both consume what it returns, and neither is
imported here.

The paper's test images ("bumps", "hairpin bend", "random", 25x25, grey levels
1-255; Sec. 3, Fig. "test images") are not available, so seeded stand-ins with
the same structure are drawn instead:

* ``blobs``: a sum of Gaussian bumps plus i.i.d. uniform noise, clipped to
  0-255 (the "bumps" stand-in, and the workload image at every size);
* ``step_edges``: half-planes lifted by a constant, added to blobs;
* ``disk_mask``: random obstacle disks until a target coverage is reached;
* ``corridor``: a dark winding corridor on a bright background (the
  "hairpin bend" stand-in);
* ``uniform_random``: i.i.d. grey levels (the "random" stand-in).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def blobs(H: int, W: int, n_blobs: int, sigma: float, noise: float, seed: int,
          amp_max: float = 200.0) -> np.ndarray:
    """Sum of ``n_blobs`` Gaussian bumps plus U(0, noise) noise, as uint8.

    Blob centres are uniform over the image, amplitudes uniform in
    [0, amp_max]; the sum is rounded to nearest and clipped to 0-255.
    """
    rng = np.random.default_rng(seed)
    return _blobs_rng(rng, H, W, n_blobs, sigma, noise, amp_max, extra=None)


def _blobs_rng(rng, H, W, n_blobs, sigma, noise, amp_max, extra):
    rr, cc = np.meshgrid(np.arange(H, dtype=np.float64),
                         np.arange(W, dtype=np.float64), indexing="ij")
    img = np.zeros((H, W), dtype=np.float64)
    mu_r = rng.uniform(0.0, H, size=n_blobs)
    mu_c = rng.uniform(0.0, W, size=n_blobs)
    amp = rng.uniform(0.0, amp_max, size=n_blobs)
    for k in range(n_blobs):
        d2 = (rr - mu_r[k]) ** 2 + (cc - mu_c[k]) ** 2
        img += amp[k] * np.exp(-d2 / (2.0 * sigma * sigma))
    if extra is not None:
        img += extra(rng, rr, cc)
    img += rng.uniform(0.0, noise, size=(H, W))
    return np.clip(np.rint(img), 0, 255).astype(np.uint8)


def blobs_with_steps(H: int, W: int, n_blobs: int, sigma: float, n_steps: int,
                     step_height: float, noise: float, seed: int) -> np.ndarray:
    """Blobs plus ``n_steps`` straight step edges, plus noise, as uint8.

    Each step edge is a half-plane through a uniform random point at a uniform
    random angle; pixels on its positive side get ``step_height`` added before
    the noise and the final clip.
    """
    rng = np.random.default_rng(seed)

    def steps(rng, rr, cc):
        out = np.zeros_like(rr)
        pr = rng.uniform(0.0, H, size=n_steps)
        pc = rng.uniform(0.0, W, size=n_steps)
        th = rng.uniform(0.0, 2.0 * math.pi, size=n_steps)
        for k in range(n_steps):
            side = (rr - pr[k]) * math.cos(th[k]) + (cc - pc[k]) * math.sin(th[k])
            out += np.where(side > 0.0, step_height, 0.0)
        return out

    return _blobs_rng(rng, H, W, n_blobs, sigma, noise, 200.0, extra=steps)


def disk_mask(H: int, W: int, coverage: float, rmin: int, rmax: int,
              seed: int) -> np.ndarray:
    """Obstacle mask: 1 = free, 0 = obstacle.

    Disks with uniform centres and integer radius uniform in [rmin, rmax] are
    added until the obstacle fraction reaches ``coverage``.
    """
    rng = np.random.default_rng(seed)
    rr, cc = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    obst = np.zeros((H, W), dtype=bool)
    target = coverage * H * W
    while obst.sum() < target:
        r0 = rng.uniform(0.0, H)
        c0 = rng.uniform(0.0, W)
        rad = int(rng.integers(rmin, rmax + 1))
        obst |= (rr - r0) ** 2 + (cc - c0) ** 2 <= rad * rad
    return (~obst).astype(np.uint8)


def uniform_random(H: int, W: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """i.i.d. grey levels uniform in [lo, hi], as uint8."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, size=(H, W)).astype(np.uint8)


def corridor(H: int, W: int, seed: int, dark: int = 5, bright: int = 220,
             noise: int = 20) -> np.ndarray:
    """A dark serpentine corridor on a bright noisy background, as uint8.

    The corridor runs along every other band of rows and turns at alternating
    ends, so geodesic paths bend back on themselves several times.
    """
    rng = np.random.default_rng(seed)
    img = np.full((H, W), bright, dtype=np.int64)
    band = max(1, H // 7)
    r = 0
    left_turn = False
    while r < H:
        img[r:r + band, 1:W - 1] = dark
        nxt = r + 2 * band
        if nxt < H:
            col = 1 if left_turn else W - 2
            img[r:nxt + band, col] = dark
        left_turn = not left_turn
        r = nxt
    img += rng.integers(0, noise + 1, size=(H, W))
    return np.clip(img, 0, 255).astype(np.uint8)


# ----------------------------------------------------------------------------
# Named workloads. Each returns a dict with the image, mask (or None), the
# connectivity, the kind ("grey" / "mask") and the batch size B.
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    img: np.ndarray
    conn: int
    kind: str = "grey"
    mask: np.ndarray | None = None
    B: int = 1
    meta: dict = field(default_factory=dict)

    @property
    def H(self) -> int:
        return int(self.img.shape[0])

    @property
    def W(self) -> int:
        return int(self.img.shape[1])

    @property
    def N(self) -> int:
        return self.H * self.W


def plain_32(seed: int = 0) -> Workload:
    """32x32, 8 blobs sigma 4, noise U(0,55), 4-connected, B=1."""
    return Workload("plain-32x32-4conn", blobs(32, 32, 8, 4.0, 55.0, seed), 4, B=1,
                    meta={"seed": seed})


def batched_128(seed: int = 0) -> Workload:
    """128x128, 32 blobs sigma 8, noise U(0,55), 8-connected, B=32."""
    return Workload("blobs-128x128-8conn-B32", blobs(128, 128, 32, 8.0, 55.0, seed),
                    8, B=32, meta={"seed": seed})


def steps_256(seed: int = 0) -> Workload:
    """256x256 blobs + 20 step edges of +100 + noise U(0,40), 8-connected."""
    img = blobs_with_steps(256, 256, 64, 16.0, 20, 100.0, 40.0, seed)
    return Workload("steps-256x256-8conn-B32", img, 8, B=32, meta={"seed": seed})


def steps_160(seed: int = 0) -> Workload:
    """The 256x256 step-edge image's generator at 160x160 (blob count and
    sigma scaled with the area and the side, 20 step edges): a smaller case
    of the same structure, for profiling."""
    img = blobs_with_steps(160, 160, 25, 10.0, 20, 100.0, 40.0, seed)
    return Workload("steps-160x160-8conn-B32", img, 8, B=32, meta={"seed": seed})


def mask_256(seed: int = 0) -> Workload:
    """256x256 obstacle disks (radius 3-12, 40% coverage), w=2, 8-connected."""
    m = disk_mask(256, 256, 0.40, 3, 12, seed)
    img = np.zeros((256, 256), dtype=np.uint8)
    return Workload("mask-256x256-8conn-B32", img, 8, kind="mask", mask=m, B=32,
                    meta={"seed": seed})


def scaled_blobs(H: int, W: int, conn: int, seed: int, B: int = 32) -> Workload:
    """Blob image of any size with the 128x128 generator's density.

    Blob count scales with area (one per 512 pixels, at least 2) and sigma
    with the mean side (8 px at 128).
    """
    nb = max(2, (H * W) // 512)
    sig = max(1.5, 8.0 * (H + W) / 256.0)
    return Workload(f"blobs-{H}x{W}-{conn}conn", blobs(H, W, nb, sig, 55.0, seed),
                    conn, B=B, meta={"seed": seed})


def batch_64(seed: int = 0, n: int = 64) -> list[Workload]:
    """Many images of uneven sizes: heights and widths log-uniform in
    [24, 96] px, drawn independently; 4- or 8-connected with equal
    probability; the blob generator at the 128x128 density; B = 32."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        H = int(round(math.exp(rng.uniform(math.log(24), math.log(96)))))
        W = int(round(math.exp(rng.uniform(math.log(24), math.log(96)))))
        conn = 4 if rng.random() < 0.5 else 8
        w = scaled_blobs(H, W, conn, seed=seed * 1000 + k, B=32)
        w.name = f"batch{k}-{H}x{W}-{conn}conn"
        out.append(w)
    return out
