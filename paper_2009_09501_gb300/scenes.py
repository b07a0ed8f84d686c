"""Seeded synthetic scenes shaped like the paper's test material.

The paper measures on 4K UHD camera photos and a 4K UHD 60 fps demo clip (Sec. 5), none
of which is available; these seeded scenes stand in for them.  This module holds none of
the pipeline's arithmetic: it only draws RGB uint8 frames, and both the CUDA path and the
CPU oracle are fed from it.

Recipe (all randomness from a counter-based SplitMix64 hash defined below, so any frame
is reproducible from (seed, frame) alone):
  * background: a vertical gradient per channel, round(lo + (hi - lo) * y / (H - 1)), with
    lo and hi uniform in 0..255;
  * objects: ellipses or rectangles (probability 1/2 each), centre uniform in the frame,
    semi-axes uniform in [W/40, W/8], base colour uniform in 0..255, drawn in index
    order (later objects cover earlier ones);
  * texture: per object, either uniform integer noise in [-32, 32] or Gaussian noise with
    sigma 8, hashed from (seed, object, local x, local y) so that it moves with the object;
  * video: each object translates by a velocity uniform in [-8, 8] px/frame with
    wrap-around, and every frame adds full-frame Gaussian noise of sigma 2 hashed from
    (seed, frame, x, y).
"""
import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)

# stream tags keep the hashed quantities of different kinds independent
_TAG_OBJ, _TAG_TEX, _TAG_FRAME, _TAG_BG = 1, 2, 3, 4


def _mix(z):
    """SplitMix64 finaliser over a uint64 array (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = z + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _C1
        z = (z ^ (z >> np.uint64(27))) * _C2
        return z ^ (z >> np.uint64(31))


def _mix_int(z):
    """The same finaliser on a Python integer."""
    m = 0xFFFFFFFFFFFFFFFF
    z = (z + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def _key(*keys):
    """Fold integer scalars into one 64-bit stream key."""
    h = 0x6A09E667F3BCC909
    for k in keys:
        h = _mix_int(h ^ (int(k) & 0xFFFFFFFFFFFFFFFF))
    return h


def _hash(key, idx):
    """Counter-based hash: one SplitMix64 round of (stream key + element counter)."""
    with np.errstate(over="ignore"):
        return _mix(np.uint64(key) + np.asarray(idx).astype(np.uint64))


def _uniform01(h):
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _gauss(key, idx):
    """Standard normal samples by Box-Muller from the two 32-bit halves of one hash."""
    h = _hash(key, idx)
    u1 = ((h >> np.uint64(40)).astype(np.float32) + np.float32(0.5)) * np.float32(1.0 / 16777216.0)
    u2 = ((h & np.uint64(0xFFFFFF)).astype(np.float32)) * np.float32(1.0 / 16777216.0)
    return np.sqrt(np.float32(-2.0) * np.log(u1)) * np.cos(np.float32(2.0 * np.pi) * u2)


def _scalar_u(seed, *keys):
    return float(_uniform01(_hash(_key(seed, _TAG_OBJ, *keys), 0)))


def _scalar_int(seed, lo, hi, *keys):
    """Uniform integer in [lo, hi]."""
    return lo + int(_scalar_u(seed, *keys) * (hi - lo + 1)) if hi > lo else lo


class Scene:
    """A seeded scene; ``frame(k)`` draws frame k as an (H, W, 3) uint8 array.

    texture: "uniform32" (uniform integer noise in [-32, 32]) or "gauss8" (sigma 8).
    moving:  objects translate between frames and per-frame sigma-2 noise is added.
    """

    def __init__(self, width, height, seed, n_objects=40, texture="gauss8", moving=False):
        self.W, self.H, self.seed = int(width), int(height), int(seed)
        self.n_objects, self.texture, self.moving = int(n_objects), texture, bool(moving)
        s, W, H = self.seed, self.W, self.H
        self.bg_lo = [_scalar_int(s, 0, 255, _TAG_BG, c, 0) for c in range(3)]
        self.bg_hi = [_scalar_int(s, 0, 255, _TAG_BG, c, 1) for c in range(3)]
        amin, amax = max(1.0, W / 40.0), max(1.0, W / 8.0)
        self.objects = []
        for i in range(self.n_objects):
            o = dict(
                ellipse=_scalar_u(s, i, 0) < 0.5,
                cx=_scalar_u(s, i, 1) * W, cy=_scalar_u(s, i, 2) * H,
                ax=amin + _scalar_u(s, i, 3) * (amax - amin),
                ay=amin + _scalar_u(s, i, 4) * (amax - amin),
                color=[_scalar_int(s, 0, 255, i, 5, c) for c in range(3)],
                vx=-8.0 + 16.0 * _scalar_u(s, i, 6), vy=-8.0 + 16.0 * _scalar_u(s, i, 7),
            )
            self.objects.append(o)

    def _background(self):
        H, W = self.H, self.W
        y = np.arange(H, dtype=np.float64)[:, None]
        frac = y / (H - 1) if H > 1 else np.zeros_like(y)
        img = np.empty((H, W, 3), np.uint8)
        for c in range(3):
            lo, hi = self.bg_lo[c], self.bg_hi[c]
            col = np.floor(lo + (hi - lo) * frac + 0.5).astype(np.uint8)
            img[:, :, c] = col
        return img

    def frame(self, k=0):
        H, W, s = self.H, self.W, self.seed
        img = self._background()
        for i, o in enumerate(self.objects):
            cx, cy = o["cx"], o["cy"]
            if self.moving:
                cx = (cx + k * o["vx"]) % W
                cy = (cy + k * o["vy"]) % H
            ax, ay = o["ax"], o["ay"]
            # draw the object and its wrapped copies so it re-enters at the other edge
            for ox in ((0.0, -W, W) if self.moving else (0.0,)):
                for oy in ((0.0, -H, H) if self.moving else (0.0,)):
                    self._paint(img, i, o, cx + ox, cy + oy, ax, ay)
        if self.moving:
            n = _gauss(_key(s, _TAG_FRAME, k), np.arange(H * W * 3, dtype=np.uint64)).reshape(H, W, 3)
            img[:] = np.clip(np.rint(img + n * np.float32(2.0)), 0, 255).astype(np.uint8)
        return img

    def _paint(self, img, i, o, cx, cy, ax, ay):
        H, W, s = self.H, self.W, self.seed
        x0, x1 = int(np.floor(cx - ax)), int(np.ceil(cx + ax)) + 1
        y0, y1 = int(np.floor(cy - ay)), int(np.ceil(cy + ay)) + 1
        bx0, bx1, by0, by1 = max(x0, 0), min(x1, W), max(y0, 0), min(y1, H)
        if bx0 >= bx1 or by0 >= by1:
            return
        yy, xx = np.mgrid[by0:by1, bx0:bx1]
        px, py = xx + 0.5 - cx, yy + 0.5 - cy
        if o["ellipse"]:
            mask = (px / ax) ** 2 + (py / ay) ** 2 <= 1.0
        else:
            mask = (np.abs(px) <= ax) & (np.abs(py) <= ay)
        if not mask.any():
            return
        # texture coordinates are local to the object so the texture moves with it
        lx = (xx[mask] - int(np.floor(cx - ax))).astype(np.int64)
        ly = (yy[mask] - int(np.floor(cy - ay))).astype(np.int64)
        # texture counter: local (x, y, channel) inside a 2^16 x 2^16 object frame
        cnt = ((ly & 0xFFFF) << 18) | ((lx & 0xFFFF) << 2)
        region = img[by0:by1, bx0:bx1]
        for c in range(3):
            key = _key(s, _TAG_TEX, i)
            if self.texture == "uniform32":
                u = _uniform01(_hash(key, cnt | c))
                n = np.floor(u * 65.0) - 32.0
            else:
                n = np.rint(_gauss(key, cnt | c) * np.float32(8.0))
            v = np.clip(o["color"][c] + n, 0, 255).astype(np.uint8)
            ch = region[:, :, c]
            ch[mask] = v


def config_scene(index, frame=0):
    """Frames of the five workloads the library is measured on, by workload number 1..5.

    1: 640x480, 12 objects, uniform-noise texture;  2: 3840x2160, 40 objects, sigma-8
    texture;  3: 3840x2160 moving video;  4 and 5 use ``batch_sizes`` / ``stream_scene``.
    """
    seed = 2009_09501 + index
    if index == 1:
        return Scene(640, 480, seed, 12, "uniform32").frame(frame)
    if index == 2:
        return Scene(3840, 2160, seed, 40, "gauss8").frame(frame)
    if index == 3:
        return Scene(3840, 2160, seed, 40, "gauss8", moving=True).frame(frame)
    raise ValueError("workloads 4 and 5 are drawn with batch_sizes() / stream_scene()")


BATCH_CLASSES = ((1280, 720), (1920, 1080), (2560, 1440), (3840, 2160), (7680, 4320))


def batch_sizes(n=64, seed=2009_09501 + 4):
    """Seeded mix of image sizes for the batched workload (classes 720p .. 8K)."""
    return [BATCH_CLASSES[_scalar_int(seed, 0, len(BATCH_CLASSES) - 1, 1000, j)] for j in range(n)]


def batch_parallax(width):
    """Maximum parallax of 2.5 % of the width (32/48/64/96/192 px for the five classes)."""
    return int(round(0.025 * width))


_POOL = {}


def batch_pool():
    """One frame per size class of the batched workload, {(W, H): (H, W, 3) uint8}: the
    images the 64-image seeded mix (batch_sizes) is made of."""
    if not _POOL:
        for i, (W, H) in enumerate(BATCH_CLASSES):
            _POOL[(W, H)] = Scene(W, H, 2009_09501 + 4 + i, 40, "gauss8").frame(0)
    return _POOL


def stream_scene(stream_index, width, height, seed=2009_09501 + 5):
    """A moving scene for one stream of the serving workload."""
    return Scene(width, height, seed * 16 + stream_index, 40, "gauss8", moving=True)
