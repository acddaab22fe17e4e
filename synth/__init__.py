"""Seeded synthetic luma sequences shaped like the paper's workloads.

This module only draws test and benchmark inputs.  It holds none of the
motion-estimation arithmetic, and both the CUDA library's tests/benchmark and
the CPU oracle receive the same frames from it.

The paper evaluates on real QCIF/CIF sequences (Sec. 4) that are not
available here; these generators stand in for them with the same frame
sizes, 8-bit luma and integer motion, plus larger frames for throughput runs.

Recipes (all frames uint8, row-major [H, W]):

* ``texture``: i.i.d. U[0,255] noise, separable Gaussian blur (sigma 1.5,
  radius 5, normalised weights, edge clamp), min-max rescaled to [16, 235],
  rounded.
* ``quadrant_sequence`` (QCIF 176x144, 10 frames): frame 0 is a texture; each
  next frame takes the previous one and pulls every destination quadrant from
  a shift (dx, dy) drawn from U{-8..8}^2 (edge clamp), adds N(0, 2^2) noise,
  rounds and clamps.
* ``global_motion_sequence`` (Sec. 3.1 set-up, default CIF): one original
  frame (``contrast_texture``: a texture times a smooth contrast map that
  runs from flat, on 30 % of the frame, to full) and nine copies displaced by known distinct global
  vectors from U{-8..8}^2 (edge clamp) plus N(0, 2^2) noise.
* ``load_sequence`` (QCIF, the Table 1-shaped load table): ``scene_sequence``
  with background contrast 0.15 or 1, 2-6 objects, object speeds up to 1 or
  3 px/frame and pans of 0-2 px/frame (``LOAD_RECIPES``); 10 fps = every
  third frame of the 30 fps scene.
* ``scene_sequence`` (CIF / 720p / 1080p / 4K): a textured background canvas
  panned by 1 px/frame, ``n_objects`` textured rectangles (sides U{32..96})
  moving at constant integer velocities from U{-vmax..vmax}^2 and painted in
  index order (clipped at the frame edge), N(0, 2^2) noise per frame, and
  optionally a fraction of block slots per frame overwritten with uniform
  noise (occlusions); frames may be padded to a taller height by repeating
  the last row.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "texture", "contrast_texture", "global_motion_sequence", "quadrant_sequence", "scene_sequence", "random_frame", "shifted_copy",
    "StreamSpec", "CONFIGS", "config_sequence", "batch_mix", "serving_mix", "LOAD_RECIPES",
    "load_sequence",
]


def _rng(*key: int) -> np.random.Generator:
    return np.random.default_rng([int(k) & 0xFFFFFFFF for k in key])


def _blur_1d(a: np.ndarray, axis: int, sigma: float, radius: int) -> np.ndarray:
    k = np.arange(-radius, radius + 1, dtype=np.float64)
    w = np.exp(-(k * k) / (2.0 * sigma * sigma))
    w /= w.sum()
    pad = [(0, 0)] * a.ndim
    pad[axis] = (radius, radius)
    ap = np.pad(a, pad, mode="edge")
    out = np.zeros_like(a, dtype=np.float64)
    n = a.shape[axis]
    for t, wt in enumerate(w):
        sl = [slice(None)] * a.ndim
        sl[axis] = slice(t, t + n)
        out += wt * ap[tuple(sl)]
    return out


def texture(rng: np.random.Generator, w: int, h: int, sigma: float = 1.5,
            radius: int = 5) -> np.ndarray:
    """Blurred uniform noise rescaled to [16, 235] (uint8, [h, w])."""
    a = rng.integers(0, 256, size=(h, w)).astype(np.float64)
    a = _blur_1d(_blur_1d(a, 1, sigma, radius), 0, sigma, radius)
    lo, hi = a.min(), a.max()
    if hi <= lo:
        return np.full((h, w), 128, np.uint8)
    a = 16.0 + (a - lo) * (219.0 / (hi - lo))
    return np.clip(np.rint(a), 0, 255).astype(np.uint8)


def _add_noise(rng: np.random.Generator, f: np.ndarray, sigma: float) -> np.ndarray:
    if sigma <= 0:
        return f.astype(np.uint8)
    g = f.astype(np.float64) + rng.normal(0.0, sigma, size=f.shape)
    return np.clip(np.rint(g), 0, 255).astype(np.uint8)


def random_frame(seed: int, w: int, h: int) -> np.ndarray:
    """Plain i.i.d. U[0,255] frame (sharp texture: every wrong shift costs a lot)."""
    return _rng(seed, 7).integers(0, 256, size=(h, w), dtype=np.uint8)


def shifted_copy(src: np.ndarray, dx: int, dy: int) -> np.ndarray:
    """dst(x, y) = src(clamp(x - dx), clamp(y - dy)): content moved by (+dx, +dy)."""
    h, w = src.shape
    xs = np.clip(np.arange(w) - dx, 0, w - 1)
    ys = np.clip(np.arange(h) - dy, 0, h - 1)
    return src[np.ix_(ys, xs)]


def quadrant_sequence(seed: int, n_frames: int = 10, w: int = 176, h: int = 144,
                      max_shift: int = 8, noise_sigma: float = 2.0) -> np.ndarray:
    """The QCIF recipe: per-quadrant integer shifts of the previous frame plus noise."""
    rng = _rng(seed, 1)
    frames = np.zeros((n_frames, h, w), np.uint8)
    frames[0] = texture(rng, w, h)
    xs = np.arange(w)
    ys = np.arange(h)
    for t in range(1, n_frames):
        prev = frames[t - 1]
        d = rng.integers(-max_shift, max_shift + 1, size=(4, 2))
        out = np.empty_like(prev)
        for q in range(4):
            qx, qy = q % 2, q // 2
            x_sl = slice(0, w // 2) if qx == 0 else slice(w // 2, w)
            y_sl = slice(0, h // 2) if qy == 0 else slice(h // 2, h)
            sx = np.clip(xs[x_sl] - d[q, 0], 0, w - 1)
            sy = np.clip(ys[y_sl] - d[q, 1], 0, h - 1)
            out[y_sl, x_sl] = prev[np.ix_(sy, sx)]
        frames[t] = _add_noise(rng, out, noise_sigma)
    return frames


def contrast_texture(rng: np.random.Generator, w: int, h: int) -> np.ndarray:
    """A texture whose local contrast varies smoothly from flat to full: the
    texture's deviation from 128 times c(x, y)^2, where c is U[0,1] noise
    blurred with sigma 12, replaced by its rank in the frame divided by the
    pixel count (uniform on [0, 1)), then mapped by max(0, (c - 0.3) / 0.7),
    so that 30 % of the frame has zero contrast (flat at 128) whatever the
    seed, and the low-contrast margin around it rounds to nearly flat."""
    t = texture(rng, w, h).astype(np.float64)
    c = rng.random((h, w))
    c = _blur_1d(_blur_1d(c, 1, 12.0, 36), 0, 12.0, 36)
    rank = np.empty(c.size, np.float64)
    rank[np.argsort(c, axis=None, kind="stable")] = np.arange(c.size)
    c = np.clip((rank.reshape(h, w) / c.size - 0.3) / 0.7, 0.0, 1.0)
    return np.clip(np.rint(128.0 + (t - 128.0) * c * c), 0, 255).astype(np.uint8)


def global_motion_sequence(seed: int, w: int = 352, h: int = 288, n_moved: int = 9,
                           max_shift: int = 8, noise_sigma: float = 2.0):
    """The known-motion set-up of Sec. 3.1: frame 0 is an original frame
    (``contrast_texture``); frames 1..n_moved are it displaced by known global
    vectors g_k drawn from U{-max_shift..max_shift}^2 without repeats, plus
    N(0, noise_sigma^2) noise.  g_k is given as the motion vector a block
    matcher should find: frame_k(x, y) = frame_0(clamp(x + gx), clamp(y + gy))
    before the noise.  Returns (frames [n_moved+1, h, w] uint8, g [n_moved, 2]
    int16 as (gx, gy))."""
    rng = _rng(seed, 11)
    base = contrast_texture(rng, w, h)
    side = 2 * max_shift + 1
    if n_moved > side * side:
        raise ValueError("more moved frames than distinct vectors")
    pick = rng.choice(side * side, size=n_moved, replace=False)
    g = np.stack([pick % side - max_shift, pick // side - max_shift], axis=1).astype(np.int16)
    frames = np.zeros((n_moved + 1, h, w), np.uint8)
    frames[0] = base
    for k in range(n_moved):
        frames[k + 1] = _add_noise(rng, shifted_copy(base, -int(g[k, 0]), -int(g[k, 1])),
                                   noise_sigma)
    return frames, g


def scene_sequence(seed: int, w: int, h: int, n_frames: int, n_objects: int = 6,
                   vmax: int = 6, pan: int = 1, noise_sigma: float = 2.0,
                   occlusion_frac: float = 0.0, block: int = 16,
                   pad_height: int | None = None, margin: int = 96,
                   bg_contrast: float = 1.0) -> np.ndarray:
    """Panned background + moving textured rectangles + noise (+ occlusion blocks).
    bg_contrast < 1 scales the background's deviation from 128 (a smoother scene)."""
    rng = _rng(seed, 2)
    cw = w + abs(pan) * n_frames + 2 * margin
    ch = h + 2 * margin
    canvas = texture(rng, cw, ch)
    if bg_contrast != 1.0:
        canvas = np.clip(np.rint(128.0 + (canvas.astype(np.float64) - 128.0) * bg_contrast),
                         0, 255).astype(np.uint8)
    objs = []
    for _ in range(n_objects):
        ow, oh = (int(v) for v in rng.integers(32, 97, size=2))
        tex = texture(rng, ow, oh)
        x0 = int(rng.integers(-ow // 2, w - ow // 2))
        y0 = int(rng.integers(-oh // 2, h - oh // 2))
        vx, vy = (int(v) for v in rng.integers(-vmax, vmax + 1, size=2))
        objs.append((tex, x0, y0, vx, vy))
    hp = h if pad_height is None else int(pad_height)
    out = np.zeros((n_frames, hp, w), np.uint8)
    for t in range(n_frames):
        ox = margin + (pan * t if pan >= 0 else abs(pan) * (n_frames - t))
        f = canvas[margin:margin + h, ox:ox + w].copy()
        for tex, x0, y0, vx, vy in objs:
            oh, ow = tex.shape
            px, py = x0 + vx * t, y0 + vy * t
            fx0, fy0 = max(px, 0), max(py, 0)
            fx1, fy1 = min(px + ow, w), min(py + oh, h)
            if fx1 <= fx0 or fy1 <= fy0:
                continue
            f[fy0:fy1, fx0:fx1] = tex[fy0 - py:fy1 - py, fx0 - px:fx1 - px]
        f = _add_noise(rng, f, noise_sigma)
        if occlusion_frac > 0:
            bw, bh = w // block, hp // block
            n_occ = int(round(occlusion_frac * bw * bh))
            slots = rng.choice(bw * bh, size=n_occ, replace=False)
            for s in slots:
                bx, by = int(s % bw), int(s // bw)
                y_lo, y_hi = by * block, min((by + 1) * block, h)
                if y_lo >= h:
                    continue
                f[y_lo:y_hi, bx * block:(bx + 1) * block] = rng.integers(
                    0, 256, size=(y_hi - y_lo, block), dtype=np.uint8)
        out[t, :h] = f
        if hp > h:
            out[t, h:] = f[h - 1]
    return out


@dataclass(frozen=True)
class StreamSpec:
    """One synthetic stream: frame size, search range and the generator seed."""
    name: str
    w: int
    h: int
    p: int
    seed: int
    n_objects: int = 6
    vmax: int = 6
    occlusion_frac: float = 0.0
    pad_height: int | None = None

    @property
    def height(self) -> int:
        return self.h if self.pad_height is None else self.pad_height


# Workload presets (frame sizes, search ranges and motion statistics).
CONFIGS = {
    "qcif": dict(w=176, h=144, p=16, frames=10, qps=(28,)),
    "cif": dict(w=352, h=288, p=16, frames=300, qps=(22, 28, 34, 40)),
    "1080p": dict(w=1920, h=1080, pad_height=1088, p=32, frames=60, qps=(28,),
                  n_objects=20, vmax=24, occlusion_frac=0.10),
}


# Four QCIF scene recipes spanning the two axes Table 1 is discussed along
# (texture of the scene, amount of motion): background contrast, objects,
# object speed bound (px per frame at 30 fps) and pan (px per frame).
LOAD_RECIPES = {
    "smooth-slow": dict(bg_contrast=0.15, n_objects=2, vmax=1, pan=0),
    "smooth-fast": dict(bg_contrast=0.15, n_objects=4, vmax=3, pan=1),
    "textured-slow": dict(bg_contrast=1.0, n_objects=4, vmax=1, pan=1),
    "textured-fast": dict(bg_contrast=1.0, n_objects=6, vmax=3, pan=2),
}


def load_sequence(name: str, fps: int, seed: int, n_frames: int = 10) -> np.ndarray:
    """QCIF frames [n_frames, 144, 176] of a ``LOAD_RECIPES`` scene at 30 fps
    (consecutive frames) or 10 fps (every third frame of the same scene, so
    three times the motion per frame)."""
    if fps not in (30, 10):
        raise ValueError("fps must be 30 or 10")
    step = 30 // fps
    r = LOAD_RECIPES[name]
    full = scene_sequence(seed, 176, 144, step * (n_frames - 1) + 1, n_objects=r["n_objects"],
                          vmax=r["vmax"], pan=r["pan"], bg_contrast=r["bg_contrast"])
    return np.ascontiguousarray(full[::step])


def config_sequence(name: str, seed: int, n_frames: int | None = None) -> np.ndarray:
    """Frames [T, H, W] of one preset (1080p comes padded to 1088 rows)."""
    c = CONFIGS[name]
    t = c["frames"] if n_frames is None else int(n_frames)
    if name == "qcif":
        return quadrant_sequence(seed, t, c["w"], c["h"])
    return scene_sequence(seed, c["w"], c["h"], t, n_objects=c.get("n_objects", 6),
                          vmax=c.get("vmax", 6), occlusion_frac=c.get("occlusion_frac", 0.0),
                          pad_height=c.get("pad_height"))


def stream_frames(spec: StreamSpec, n_frames: int) -> np.ndarray:
    return scene_sequence(spec.seed, spec.w, spec.h, n_frames, n_objects=spec.n_objects,
                          vmax=spec.vmax, occlusion_frac=spec.occlusion_frac,
                          pad_height=spec.pad_height)


def batch_mix(base_seed: int = 1000) -> list[StreamSpec]:
    """64 uneven streams: 24 QCIF p16, 24 CIF p16, 12 720p p32, 4 2160p p64."""
    specs = []
    sizes = [("qcif", 176, 144, 16, 24), ("cif", 352, 288, 16, 24),
             ("720p", 1280, 720, 32, 12), ("2160p", 3840, 2160, 64, 4)]
    for name, w, h, p, n in sizes:
        for _ in range(n):
            specs.append(StreamSpec(name, w, h, p, base_seed + len(specs)))
    return specs


def serving_mix(n_streams: int = 200, seed: int = 5000) -> list[StreamSpec]:
    """Streams drawn CIF p16 : 720p p32 : 1080p p32 = 50 : 35 : 15."""
    rng = _rng(seed, 3)
    kinds = [("cif", 352, 288, 16, None), ("720p", 1280, 720, 32, None),
             ("1080p", 1920, 1080, 32, 1088)]
    pick = rng.choice(3, size=n_streams, p=[0.50, 0.35, 0.15])
    specs = []
    for i, k in enumerate(pick):
        name, w, h, p, ph = kinds[int(k)]
        specs.append(StreamSpec(name, w, h, p, seed + 1 + i, pad_height=ph))
    return specs
