"""Seeded synthetic inputs for the bilateral solver workloads.

This module only draws random inputs; it holds none of the solver's
arithmetic, so both the CUDA path and the CPU oracle may use it.

Inputs follow the structure of the paper's applications (Sec. 4): a
reference RGB image converted to YUV (the affinity of Eq. (2) is measured in
YUV), a per-pixel target t and a per-pixel confidence c.  The reference
images are flat-coloured random polygons plus Gaussian noise; targets are
piecewise-planar per polygon (stereo / depth), chroma of the clean image
(colourisation) or softmax probabilities over smooth label blobs
(segmentation).  Every generator is driven by numpy's PCG64 with an explicit
seed.

YUV reading: the paper does not name the matrix (Sec. 2, footnote on luma);
we use full-range BT.601 (JPEG), which keeps every coordinate >= 0.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np


def rgb_to_yuv_planar(rgb: np.ndarray) -> np.ndarray:
    """uint8 H x W x 3 RGB -> float32 planar 3 x H x W (l, u, v), computed in FP64."""
    f = rgb.astype(np.float64)
    r, g, b = f[..., 0], f[..., 1], f[..., 2]
    y = 0.299 * r + 0.587 * g + 0.114 * b
    u = 128.0 - 0.168736 * r - 0.331264 * g + 0.5 * b
    v = 128.0 + 0.5 * r - 0.418688 * g - 0.081312 * b
    return np.stack([y, u, v]).astype(np.float32)


def _polygon_mask(h: int, w: int, px: np.ndarray, py: np.ndarray):
    """Even-odd point-in-polygon test for pixel centres (x, y) on the bounding box.

    Returns (y0, y1, x0, x1, mask) with mask of shape (y1-y0, x1-x0)."""
    x0 = max(int(np.floor(px.min())), 0)
    x1 = min(int(np.ceil(px.max())) + 1, w)
    y0 = max(int(np.floor(py.min())), 0)
    y1 = min(int(np.ceil(py.max())) + 1, h)
    if x0 >= x1 or y0 >= y1:
        return 0, 0, 0, 0, None
    ys = np.arange(y0, y1, dtype=np.float64)[:, None]
    xs = np.arange(x0, x1, dtype=np.float64)[None, :]
    inside = np.zeros((y1 - y0, x1 - x0), dtype=bool)
    n = len(px)
    for k in range(n):
        xa, ya = px[k], py[k]
        xb, yb = px[(k + 1) % n], py[(k + 1) % n]
        if ya == yb:
            continue
        crosses = (ya > ys) != (yb > ys)
        xcross = xa + (ys - ya) * (xb - xa) / (yb - ya)
        inside ^= crosses & (xs < xcross)
    return y0, y1, x0, x1, inside


def polygon_scene(rng: np.random.Generator, h: int, w: int, n_polygons: int):
    """Flat-coloured random star-shaped polygons over a random background.

    Returns (rgb_clean uint8 HxWx3, labels int32 HxW with 0 = background,
    centres float64 (n_polygons+1) x 2)."""
    bg = rng.integers(0, 256, size=3)
    rgb = np.empty((h, w, 3), dtype=np.uint8)
    rgb[:] = bg
    labels = np.zeros((h, w), dtype=np.int32)
    centres = np.zeros((n_polygons + 1, 2))
    centres[0] = (w / 2.0, h / 2.0)
    rmax = 0.5 * min(h, w)
    for i in range(n_polygons):
        nv = int(rng.integers(3, 9))
        cx = rng.uniform(0, w)
        cy = rng.uniform(0, h)
        ang = np.sort(rng.uniform(0.0, 2.0 * np.pi, size=nv))
        scale = rng.uniform(0.15, 1.0) * rmax
        rad = scale * rng.uniform(0.3, 1.0, size=nv)
        px = cx + rad * np.cos(ang)
        py = cy + rad * np.sin(ang)
        colour = rng.integers(0, 256, size=3)
        centres[i + 1] = (cx, cy)
        y0, y1, x0, x1, m = _polygon_mask(h, w, px, py)
        if m is None:
            continue
        rgb[y0:y1, x0:x1][m] = colour
        labels[y0:y1, x0:x1][m] = i + 1
    return rgb, labels, centres


def add_noise_u8(rng: np.random.Generator, rgb: np.ndarray, sigma: float) -> np.ndarray:
    """Add N(0, sigma^2) per channel, round, clip to uint8."""
    noisy = rgb.astype(np.float64) + rng.normal(0.0, sigma, size=rgb.shape)
    return np.clip(np.rint(noisy), 0, 255).astype(np.uint8)


def planar_target(rng: np.random.Generator, labels: np.ndarray, centres: np.ndarray,
                  noise_sigma: float) -> np.ndarray:
    """One plane per label: z = a (x - x0) + b (y - y0) + z0, clipped to [0, 255], + noise."""
    h, w = labels.shape
    nl = centres.shape[0]
    z0 = rng.uniform(0.0, 255.0, size=nl)
    slope = 128.0 / max(h, w)
    a = rng.uniform(-1.0, 1.0, size=nl) * slope
    b = rng.uniform(-1.0, 1.0, size=nl) * slope
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    lab = labels
    z = a[lab] * (xs - centres[lab, 0]) + b[lab] * (ys - centres[lab, 1]) + z0[lab]
    z = np.clip(z, 0.0, 255.0)
    if noise_sigma > 0:
        z = z + rng.normal(0.0, noise_sigma, size=z.shape)
    return z.astype(np.float32)


@dataclasses.dataclass
class Instance:
    """One image of a workload: reference, target and confidence plus parameters."""
    yuv: np.ndarray          # float32 3 x H x W (l, u, v)
    t: np.ndarray            # float32 C x H x W
    c: np.ndarray            # float32 H x W
    sigma_xy: float
    sigma_l: float
    sigma_uv: float
    lam: float
    label: Optional[np.ndarray] = None   # float32 C x H x W (segmentation loss target)

    @property
    def height(self) -> int:
        return int(self.yuv.shape[1])

    @property
    def width(self) -> int:
        return int(self.yuv.shape[2])

    @property
    def channels(self) -> int:
        return int(self.t.shape[0])

    @property
    def n_pixels(self) -> int:
        return self.height * self.width


def depth_instance(rng, h, w, n_polygons, sigmas, lam, channels=1, noise_sigma=8.0):
    """Polygon reference with piecewise-planar target(s) and c ~ U[0, 1]."""
    rgb, labels, centres = polygon_scene(rng, h, w, n_polygons)
    yuv = rgb_to_yuv_planar(add_noise_u8(rng, rgb, 4.0))
    t = np.stack([planar_target(rng, labels, centres, noise_sigma) for _ in range(channels)])
    c = rng.uniform(0.0, 1.0, size=(h, w)).astype(np.float32)
    return Instance(yuv, t, c, *sigmas, lam)


def robust_instance(rng, h, w, n_polygons, sigmas, lam, outlier_frac=0.05, mask_frac=0.10):
    """Noise-free planar disparity with uniform outliers; c_init = 0 on a random mask."""
    rgb, labels, centres = polygon_scene(rng, h, w, n_polygons)
    yuv = rgb_to_yuv_planar(add_noise_u8(rng, rgb, 4.0))
    t = planar_target(rng, labels, centres, 0.0)
    out = rng.random((h, w)) < outlier_frac
    t[out] = rng.uniform(0.0, 255.0, size=int(out.sum())).astype(np.float32)
    c = np.ones((h, w), dtype=np.float32)
    c[rng.random((h, w)) < mask_frac] = 0.0
    return Instance(yuv, t[None], c, *sigmas, lam)


def chroma_instance(rng, h, w, n_polygons, sigmas, lam, hint_frac=0.02):
    """Colourisation-style: grey reference, target = true (u, v), c = 1 on sparse hints."""
    rgb, _, _ = polygon_scene(rng, h, w, n_polygons)
    yuv_true = rgb_to_yuv_planar(rgb)
    grey = add_noise_u8(rng, np.repeat(np.clip(np.rint(yuv_true[0]), 0, 255)
                                       .astype(np.uint8)[..., None], 3, axis=2), 4.0)
    yuv = np.stack([grey[..., 0].astype(np.float32),
                    np.full((h, w), 128.0, np.float32),
                    np.full((h, w), 128.0, np.float32)])
    t = yuv_true[1:3].copy()
    c = (rng.random((h, w)) < hint_frac).astype(np.float32)
    return Instance(yuv, t, c, *sigmas, lam)


def _smooth(field: np.ndarray, sigma: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(field, sigma=sigma, mode="reflect")


def _smooth_stack(fields: np.ndarray, sigma: float) -> np.ndarray:
    """Smooth each 2-D slice of a stack (no smoothing across the first axis)."""
    from scipy.ndimage import gaussian_filter
    return gaussian_filter(fields, sigma=(0.0, sigma, sigma), mode="reflect", truncate=3.0)


def _smooth_field(rng, h, w, sigma, step=8):
    """Gaussian-smoothed white noise, drawn on a grid `step` times coarser and
    bilinearly upsampled (the field is smooth on that scale anyway)."""
    from scipy.ndimage import zoom
    hs, ws = max(2, -(-h // step) + 1), max(2, -(-w // step) + 1)
    coarse = _smooth(rng.normal(size=(hs, ws)), sigma / step)
    return zoom(coarse, (h / hs, w / ws), order=1)[:h, :w]


def segmentation_instance(rng, h, w, n_classes, sigmas, lam, blob_sigma=24.0, n_present=None):
    """Label blobs = argmax over smoothed random fields; t = softmax of smoothed noisy logits.

    With n_present, only that many classes (drawn at random) occur in the
    label map and the others get logits 8 lower (probability ~3e-4 of a
    present class's), as a CNN assigns next to nothing to classes absent
    from a scene: B = S(c o t) is then close to rank n_present."""
    step = 8 if blob_sigma >= 16 else 1
    fields = np.stack([_smooth_field(rng, h, w, blob_sigma, step) for _ in range(n_classes)])
    absent = None
    if n_present is not None:
        present = rng.choice(n_classes, size=n_present, replace=False)
        absent = np.ones(n_classes, bool)
        absent[present] = False
        fields[absent] = -np.inf
    labels = np.argmax(fields, axis=0)
    colours = rng.integers(0, 256, size=(n_classes, 3))
    rgb = colours[labels].astype(np.uint8)
    yuv = rgb_to_yuv_planar(add_noise_u8(rng, rgb, 4.0))
    onehot = (labels[None] == np.arange(n_classes)[:, None, None]).astype(np.float64)
    logits = 4.0 * onehot + rng.normal(size=onehot.shape)
    if absent is not None:
        logits[absent] -= 8.0
    logits = _smooth_stack(logits, 2.0)
    logits -= logits.max(axis=0, keepdims=True)
    e = np.exp(logits)
    t = (e / e.sum(axis=0, keepdims=True)).astype(np.float32)
    c = rng.uniform(0.0, 1.0, size=(h, w)).astype(np.float32)
    # seeded perturbation of the label map for the loss target
    dy, dx = int(rng.integers(-3, 4)), int(rng.integers(-3, 4))
    lab2 = np.roll(np.roll(labels, dy, axis=0), dx, axis=1)
    label = (lab2[None] == np.arange(n_classes)[:, None, None]).astype(np.float32)
    return Instance(yuv, t, c, *sigmas, lam, label=label)


def make_tiny(seed: int, h: int, w: int, n_polygons: int = 3, channels: int = 1,
              sigmas=(8.0, 4.0, 3.0), lam: float = 128.0, noise_sigma: float = 8.0) -> Instance:
    """A small depth-style instance for pins and parity tests."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return depth_instance(rng, h, w, n_polygons, sigmas, lam, channels, noise_sigma)


@dataclasses.dataclass
class Workload:
    name: str
    instances: List[Instance]
    bistoch_iters: int = 2
    pcg_iters: int = 25
    irls_iters: int = 0
    sigma_gm: float = 1.0
    backward: bool = False

    @property
    def n_pixels(self) -> int:
        return sum(i.n_pixels for i in self.instances)


def plain_64x48(seed: int = 1) -> Workload:
    """One 64x48 image, 6 polygons, C = 1, sigma = (8, 4, 3), lambda = 128."""
    rng = np.random.Generator(np.random.PCG64(seed))
    inst = depth_instance(rng, 48, 64, 6, (8.0, 4.0, 3.0), 128.0, 1)
    return Workload("plain 64x48 C=1", [inst])


def plain_1080p(seed: int = 2, h: int = 1080, w: int = 1920) -> Workload:
    """One 1920x1080 image, 40 polygons, C = 3, sigma = (16, 8, 8), lambda = 128."""
    rng = np.random.Generator(np.random.PCG64(seed))
    inst = depth_instance(rng, h, w, 40, (16.0, 8.0, 8.0), 128.0, 3)
    return Workload(f"plain {w}x{h} C=3", [inst])


def robust_1400x1000(seed: int = 3, h: int = 1000, w: int = 1400) -> Workload:
    """Geman-McClure RBS on a 1400x1000 planar disparity with 5 % outliers.

    Parameters are the paper's Middlebury RBS settings (supplement Sec. 5.1):
    sigma_xy = sigma_l = sigma_uv = 4, lambda = 0.25, sigma_gm = 1; 10 IRLS x 25 PCG."""
    rng = np.random.Generator(np.random.PCG64(seed))
    inst = robust_instance(rng, h, w, 40, (4.0, 4.0, 4.0), 0.25)
    return Workload(f"robust {w}x{h} C=1", [inst], irls_iters=10, sigma_gm=1.0)


def batched_64(seed: int = 4, n_images: int = 64, max_hw=(1080, 1920), min_hw=(240, 320)) -> Workload:
    """64 images of uneven size; half depth (C = 1), half chroma (C = 2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    insts = []
    amin = min_hw[0] * min_hw[1]
    amax = max_hw[0] * max_hw[1]
    for _ in range(n_images):
        w = int(rng.integers(min_hw[1], max_hw[1] + 1))
        h = int(rng.integers(min_hw[0], max_hw[0] + 1))
        frac = (h * w - amin) / max(amax - amin, 1)
        npoly = int(round(6 + 34 * min(max(frac, 0.0), 1.0)))
        sxy = float(rng.choice([8.0, 16.0]))
        sig = (8.0, 4.0, 3.0) if sxy == 8.0 else (16.0, 8.0, 8.0)
        lam = float(rng.choice([32.0, 128.0]))
        if rng.random() < 0.5:
            insts.append(depth_instance(rng, h, w, npoly, sig, lam, 1))
        else:
            insts.append(chroma_instance(rng, h, w, npoly, sig, lam))
    return Workload(f"batched {n_images} images", insts)


def segmentation_16(seed: int = 5, n_images: int = 16, h: int = 480, w: int = 640) -> Workload:
    """16 images 640x480, C = 21 softmax targets, c ~ U[0, 1]; forward + backward."""
    rng = np.random.Generator(np.random.PCG64(seed))
    insts = [segmentation_instance(rng, h, w, 21, (8.0, 4.0, 3.0), 128.0) for _ in range(n_images)]
    return Workload(f"segmentation {n_images}x{w}x{h} C=21", insts, backward=True)


def segmentation_scenes_16(seed: int = 6, n_images: int = 16, h: int = 480, w: int = 640,
                           n_present=(2, 6)) -> Workload:
    """16 images 640x480, C = 21 softmax targets of which 2-6 classes occur
    per image (the regime of the low-rank reduction), c ~ U[0, 1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    insts = [segmentation_instance(rng, h, w, 21, (8.0, 4.0, 3.0), 128.0,
                                   n_present=int(rng.integers(n_present[0], n_present[1] + 1)))
             for _ in range(n_images)]
    return Workload(f"segmentation scenes {n_images}x{w}x{h} C=21", insts)


def crop(inst: Instance, y0: int, x0: int, h: int, w: int) -> Instance:
    """A sub-window of an instance (for finite-difference checks)."""
    sl = (slice(y0, y0 + h), slice(x0, x0 + w))
    lab = None if inst.label is None else np.ascontiguousarray(inst.label[:, sl[0], sl[1]])
    return Instance(np.ascontiguousarray(inst.yuv[:, sl[0], sl[1]]),
                    np.ascontiguousarray(inst.t[:, sl[0], sl[1]]),
                    np.ascontiguousarray(inst.c[sl]),
                    inst.sigma_xy, inst.sigma_l, inst.sigma_uv, inst.lam, lab)
