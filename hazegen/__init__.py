"""Seeded synthetic hazy frames.

This module only makes inputs. It draws a clear scene J, a depth map d and an
airlight A from a seeded PCG64 stream, and renders the hazy observation with
the forward scattering model I = J*t + A*(1-t), t = exp(-beta*d) (Section III,
Eq. 1). It contains none of the dehazing method (dark channel, airlight
estimate, transmission, reconstruction, gamma, balance, guided filter), so
that both the CPU oracle and the GPU tests can draw the same frames from it
without sharing any of the method's arithmetic.

Scene recipe (resolution independent: a seed gives the same scene at any size):

* J, per channel: 12 isotropic Gaussian blobs (centres uniform over the frame,
  sigma = U(0.05, 0.25) * min(W, H), amplitude U(0, 1)), min-max normalised to
  [0, 1]; then 8 sharp axis-aligned rectangles of size U(0.05, 0.3) * (W, H)
  with colour U(0, 1)^3, one random channel of each set to U(0, 0.1) so that
  the dark-channel prior holds inside them.
* d: a vertical gradient 2.4 * (1 - y / (H - 1)) (far at the top), then 3
  rectangles with planar depth a + b*x_n + c*y_n merged by minimum, clipped to
  [0, 3]. In a sequence the rectangles drift at a constant per-rectangle
  velocity of at most 2 px/frame.
* A = (0.85, 0.88, 0.90) + U(-0.03, 0.03)^3.
* I = J*t + A*(1 - t) (evaluated as A + (J - A)*t) in float64, quantised as
  clip(rint(255*I), 0, 255) to
  uint8, RGB interleaved (H, W, 3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Scene",
    "make_scene",
    "render",
    "make_frame",
    "make_sequence",
    "sequence_beta",
    "mixed_batch_specs",
    "random_u8_image",
    "rgb_to_nv12",
]

BASE_AIRLIGHT = (0.85, 0.88, 0.90)


@dataclass
class Scene:
    """A drawn scene: clear radiance, depth planes and airlight."""

    W: int
    H: int
    J: np.ndarray  # (H, W, 3) float64 in [0, 1]
    A: np.ndarray  # (3,) float64
    planes: list  # [(x0, y0, w, h, a, b, c, vx, vy)] in pixels / normalised coeffs


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def make_scene(W: int, H: int, seed: int) -> Scene:
    """Draw the clear scene, the depth rectangles and the airlight."""
    if W < 1 or H < 1:
        raise ValueError("W and H must be >= 1")
    g = _rng(seed)
    xs = np.arange(W, dtype=np.float64) + 0.5
    ys = np.arange(H, dtype=np.float64) + 0.5
    J = np.zeros((H, W, 3), dtype=np.float64)
    smin = float(min(W, H))
    for c in range(3):
        acc = np.zeros((H, W), dtype=np.float64)
        for _ in range(12):
            cx, cy = g.uniform(0.0, 1.0, size=2)
            sig = g.uniform(0.05, 0.25) * smin
            amp = g.uniform(0.0, 1.0)
            gx = np.exp(-((xs - cx * W) ** 2) / (2.0 * sig * sig))
            gy = np.exp(-((ys - cy * H) ** 2) / (2.0 * sig * sig))
            acc += amp * np.outer(gy, gx)
        lo, hi = acc.min(), acc.max()
        J[:, :, c] = (acc - lo) / (hi - lo) if hi > lo else 0.0
    for _ in range(8):
        rw = max(1, int(round(g.uniform(0.05, 0.3) * W)))
        rh = max(1, int(round(g.uniform(0.05, 0.3) * H)))
        x0 = int(g.integers(0, max(1, W - rw + 1)))
        y0 = int(g.integers(0, max(1, H - rh + 1)))
        col = g.uniform(0.0, 1.0, size=3)
        col[int(g.integers(0, 3))] = g.uniform(0.0, 0.1)
        J[y0:y0 + rh, x0:x0 + rw, :] = col
    planes = []
    for _ in range(3):
        pw = max(1, int(round(g.uniform(0.1, 0.4) * W)))
        ph = max(1, int(round(g.uniform(0.1, 0.4) * H)))
        px = float(g.integers(0, max(1, W - pw + 1)))
        py = float(g.integers(0, max(1, H - ph + 1)))
        a = g.uniform(0.2, 1.5)
        b = g.uniform(-0.5, 0.5)
        c = g.uniform(-0.5, 0.5)
        ang = g.uniform(0.0, 2.0 * math.pi)
        spd = g.uniform(0.0, 2.0)
        planes.append((px, py, pw, ph, a, b, c, spd * math.cos(ang), spd * math.sin(ang)))
    A = np.array(BASE_AIRLIGHT, dtype=np.float64) + g.uniform(-0.03, 0.03, size=3)
    return Scene(W=W, H=H, J=J, A=A, planes=planes)


def _depth(scene: Scene, frame: int) -> np.ndarray:
    W, H = scene.W, scene.H
    yy = np.arange(H, dtype=np.float64)
    grad = 2.4 * (1.0 - yy / max(H - 1, 1))
    d = np.repeat(grad[:, None], W, axis=1)
    for (px, py, pw, ph, a, b, c, vx, vy) in scene.planes:
        x0 = int(round(px + vx * frame))
        y0 = int(round(py + vy * frame))
        xa, xb = max(0, x0), min(W, x0 + pw)
        ya, yb = max(0, y0), min(H, y0 + ph)
        if xa >= xb or ya >= yb:
            continue
        xn = (np.arange(xa, xb, dtype=np.float64) + 0.5) / W
        yn = (np.arange(ya, yb, dtype=np.float64) + 0.5) / H
        plane = a + b * xn[None, :] + c * yn[:, None]
        np.minimum(d[ya:yb, xa:xb], plane, out=d[ya:yb, xa:xb])
    return np.clip(d, 0.0, 3.0)


def render(scene: Scene, beta: float, frame: int = 0, with_truth: bool = False):
    """Render one hazy uint8 frame (H, W, 3) of the scene (Eq. 1 forward)."""
    d = _depth(scene, frame)
    t = np.exp(-beta * d)
    # I = J t + A (1 - t), evaluated as A + (J - A) t in place
    I = scene.J - scene.A
    I *= t[:, :, None]
    I += scene.A
    I *= 255.0
    np.rint(I, out=I)
    np.clip(I, 0, 255, out=I)
    u8 = I.astype(np.uint8)
    if with_truth:
        return u8, {"J": scene.J, "t": t, "A": scene.A.copy(), "d": d}
    return u8


def make_frame(W: int, H: int, seed: int, beta: float = 1.0, with_truth: bool = False):
    """One hazy frame from a fresh scene."""
    return render(make_scene(W, H, seed), beta, 0, with_truth)


def sequence_beta(f: int, n: int = 300) -> float:
    """Haze density of frame f of a sequence: 1 + 0.4 sin(2 pi f / n)."""
    return 1.0 + 0.4 * math.sin(2.0 * math.pi * f / n)


def make_sequence(W: int, H: int, n_frames: int, seed: int, period: int = 300,
                  out: np.ndarray | None = None) -> np.ndarray:
    """(n_frames, H, W, 3) uint8: drifting depth rectangles, sinusoidal beta."""
    scene = make_scene(W, H, seed)
    if out is None:
        out = np.empty((n_frames, H, W, 3), dtype=np.uint8)
    for f in range(n_frames):
        out[f] = render(scene, sequence_beta(f, period), f)
    return out


def mixed_batch_specs(n_per_size: int = 16, seed: int = 100):
    """(W, H, seed, beta) for the mixed-size batch: n each of 854x480,
    1280x720, 1920x1080, 3840x2160, beta ~ U(0.5, 1.5)."""
    g = _rng(seed)
    sizes = [(854, 480), (1280, 720), (1920, 1080), (3840, 2160)]
    specs = []
    i = 0
    for (W, H) in sizes:
        for _ in range(n_per_size):
            specs.append((W, H, seed + i, float(g.uniform(0.5, 1.5))))
            i += 1
    return specs


def random_u8_image(W: int, H: int, seed: int, levels: int = 256) -> np.ndarray:
    """Unstructured uint8 RGB noise (H, W, 3) with values in [0, levels)."""
    g = _rng(seed)
    return g.integers(0, levels, size=(H, W, 3), dtype=np.uint8)


def rgb_to_nv12(I: np.ndarray) -> np.ndarray:
    """A camera-style NV12 frame (3H/2, W) uint8 from an RGB frame (H, W, 3)
    with even sizes: BT.601 limited-range forward transform in float
    (Y = 16 + 65.481 R + 128.553 G + 24.966 B, Cb = 128 - 37.797 R - 74.203 G
    + 112 B, Cr = 128 + 112 R - 93.786 G - 18.214 B on R, G, B in [0, 1]),
    chroma averaged over 2 x 2 blocks, rounded and clipped; the luma rows,
    then the interleaved Cb/Cr rows."""
    H, W, _ = I.shape
    if H % 2 or W % 2:
        raise ValueError("NV12 needs even W and H")
    x = I.astype(np.float64) / 255.0
    R, G, B = x[..., 0], x[..., 1], x[..., 2]
    Y = 16 + 65.481 * R + 128.553 * G + 24.966 * B
    Cb = 128 - 37.797 * R - 74.203 * G + 112.0 * B
    Cr = 128 + 112.0 * R - 93.786 * G - 18.214 * B
    Cb = Cb.reshape(H // 2, 2, W // 2, 2).mean(axis=(1, 3))
    Cr = Cr.reshape(H // 2, 2, W // 2, 2).mean(axis=(1, 3))
    out = np.empty((H + H // 2, W), np.uint8)
    out[:H] = np.clip(np.rint(Y), 0, 255)
    uv = np.stack([Cb, Cr], axis=-1).reshape(H // 2, W)
    out[H:] = np.clip(np.rint(uv), 0, 255)
    return out
