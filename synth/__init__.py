"""Seeded synthetic inputs shared by the CPU oracle, the tests and the bench.

This module only draws pseudo-random search images and templates; it holds
none of the template-search arithmetic (no correlation, no bounds, no blur
decisions).  Every generator takes an explicit seed and uses numpy's PCG64
(`numpy.random.default_rng`).

Workloads (stand-ins for the paper's satellite/aerial datasets, which are
not available; the paper's experiments, Section 7, use real 962x622 and
1549x2389 images with square templates of 21..129 pixels):

* ``white_blur_image``  -- white Gaussian noise smoothed with a Gaussian of
  sigma 2, rescaled to [0, 255] and rounded to integers (float32).
* ``aerial_image``      -- "remote-sensing-like" uint8 image: 1/f multi-octave
  value noise (bilinearly upsampled random grids, one per octave, all with
  the same amplitude: a 1/f amplitude spectrum puts equal variance in every
  octave of a 2-D image, the statistic of natural and aerial images) plus
  axis-aligned rectangles and line segments of random intensity, rescaled
  to [0, 255] and rounded.
* ``make_templates``    -- square crops of the search image at seeded
  locations, transformed by an affine intensity map a*x+b and perturbed by
  additive Gaussian noise (float32); with ``quantize`` rounded and clipped
  to 0..255 like an 8-bit photograph, as the named workloads are (the
  paper's templates are images taken from another view at another time),
  else left as real values (not clipped).
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "white_blur_image", "aerial_image", "make_templates", "Template",
    "WORKLOADS", "workload_image", "workload_templates", "BATCH_SIZES",
    "aerial_image_device", "SERVE_IMAGES", "serve_image",
]

# Square template sizes of the uneven-size batch (4096^2 image, 256 templates).
BATCH_SIZES = (16, 24, 32, 48, 64, 96, 128)


@dataclasses.dataclass
class Template:
    data: np.ndarray          # float32 (m, n), C-contiguous
    y: int                    # top-left row of the crop it was made from
    x: int                    # top-left column of the crop
    a: float                  # intensity gain
    b: float                  # intensity offset
    noise: float              # additive noise std


def _rescale_round(x: np.ndarray) -> np.ndarray:
    lo, hi = float(x.min()), float(x.max())
    if hi <= lo:
        return np.zeros(x.shape, dtype=np.float32)
    y = (x - lo) * (255.0 / (hi - lo))
    return np.rint(y).astype(np.float32)


def white_blur_image(size: int = 256, seed: int = 1001, sigma: float = 2.0) -> np.ndarray:
    """White N(0,1) noise -> Gaussian smoothing (sigma, radius 3*sigma,
    reflect borders) -> linear rescale to [0,255] -> rint.  float32."""
    from scipy import ndimage  # library smoothing, used for input synthesis only
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((size, size))
    s = ndimage.gaussian_filter(w, sigma=sigma, mode="reflect", truncate=3.0)
    return _rescale_round(s)


def _upsample_bilinear(grid: np.ndarray, rows: int, cols: int) -> np.ndarray:
    """Cell-centred bilinear upsampling of a small grid to rows x cols (float32)."""
    gr, gc = grid.shape
    yr = (np.arange(rows, dtype=np.float64) + 0.5) * (gr / rows) - 0.5
    xc = (np.arange(cols, dtype=np.float64) + 0.5) * (gc / cols) - 0.5
    yr = np.clip(yr, 0, gr - 1)
    xc = np.clip(xc, 0, gc - 1)
    y0 = np.floor(yr).astype(np.int64); y1 = np.minimum(y0 + 1, gr - 1); fy = (yr - y0).astype(np.float32)
    x0 = np.floor(xc).astype(np.int64); x1 = np.minimum(x0 + 1, gc - 1); fx = (xc - x0).astype(np.float32)
    g = grid.astype(np.float32)
    # interpolate along columns first (small), then rows
    gx = g[:, x0] * (1.0 - fx)[None, :] + g[:, x1] * fx[None, :]          # (gr, cols)
    out = gx[y0, :] * (1.0 - fy)[:, None] + gx[y1, :] * fy[:, None]        # (rows, cols)
    return out.astype(np.float32, copy=False)


def _draw_segment(img: np.ndarray, y0, x0, y1, x1, width, amp):
    rows, cols = img.shape
    r = width / 2.0 + 1.0
    ymin = int(max(0, np.floor(min(y0, y1) - r))); ymax = int(min(rows, np.ceil(max(y0, y1) + r) + 1))
    xmin = int(max(0, np.floor(min(x0, x1) - r))); xmax = int(min(cols, np.ceil(max(x0, x1) + r) + 1))
    if ymin >= ymax or xmin >= xmax:
        return
    yy, xx = np.mgrid[ymin:ymax, xmin:xmax].astype(np.float32)
    dy, dx = y1 - y0, x1 - x0
    L2 = dy * dy + dx * dx
    tpar = ((yy - y0) * dy + (xx - x0) * dx) / max(L2, 1e-12)
    tpar = np.clip(tpar, 0.0, 1.0)
    py, px = y0 + tpar * dy, x0 + tpar * dx
    d2 = (yy - py) ** 2 + (xx - px) ** 2
    mask = d2 <= (width / 2.0) ** 2
    img[ymin:ymax, xmin:xmax][mask] += amp


def aerial_image(size: int, n_octaves: int, n_prims: int, seed: int,
                 as_float32: bool = False, decay: float = 1.0) -> np.ndarray:
    """Remote-sensing-like image, uint8 (or float32 holding the same integers).

    1/f noise: octave o = 0..n_octaves-1 is an N(0,1) grid of
    (size / 2**(n_octaves-o))**2 cells -- the finest octave has 2-pixel cells --
    bilinearly upsampled to size x size and scaled by decay**o (decay = 1:
    equal variance per octave, a 1/f amplitude spectrum; decay = 0.5 gives
    the much smoother "persistence 1/2" fractal sum).  Then n_prims
    primitives, half axis-aligned rectangles (sides U{8..256}) and half line
    segments (length U{32..512}, width U{1..3}, uniform angle), each added
    with amplitude U[-3,3] * std(noise).  Rescaled to [0,255], rounded.
    """
    rng = np.random.default_rng(seed)
    acc = np.zeros((size, size), dtype=np.float32)
    for o in range(n_octaves):
        cells = max(2, size >> (n_octaves - o))
        grid = rng.standard_normal((cells, cells))
        acc += _upsample_bilinear(grid, size, size) * np.float32(decay ** o)
    sd = float(acc.std())
    n_rect = n_prims // 2
    for _ in range(n_rect):
        hgt = int(rng.integers(8, 257)); wid = int(rng.integers(8, 257))
        y = int(rng.integers(0, size)); x = int(rng.integers(0, size))
        amp = float(rng.uniform(-3.0, 3.0)) * sd
        acc[y:min(size, y + hgt), x:min(size, x + wid)] += np.float32(amp)
    for _ in range(n_prims - n_rect):
        length = float(rng.integers(32, 513)); width = float(rng.integers(1, 4))
        ang = float(rng.uniform(0.0, np.pi))
        y0 = float(rng.uniform(0, size)); x0 = float(rng.uniform(0, size))
        y1 = y0 + length * np.sin(ang); x1 = x0 + length * np.cos(ang)
        amp = float(rng.uniform(-3.0, 3.0)) * sd
        _draw_segment(acc, np.float32(y0), np.float32(x0), np.float32(y1), np.float32(x1),
                      width, np.float32(amp))
    out = _rescale_round(acc)
    return out if as_float32 else out.astype(np.uint8)


def aerial_image_device(size: int, n_octaves: int, n_prims: int, seed: int, device="cuda"):
    """``aerial_image``'s recipe drawn on a torch device, for images too large
    to draw quickly on the host (uint8 tensor of size x size on `device`).

    Every random number comes from the same numpy PCG64 stream in the same
    order as ``aerial_image``; the upsampling (bilinear, cell-centred, edge
    clamped), the primitives and the final rescale run in float32 on the
    device, so a pixel may differ by one grey level from the host version
    where float rounding lands on a rounding boundary.  Octave amplitudes
    are equal (decay 1)."""
    import torch
    import torch.nn.functional as F
    rng = np.random.default_rng(seed)
    acc = torch.zeros((size, size), dtype=torch.float32, device=device)
    for o in range(n_octaves):
        cells = max(2, size >> (n_octaves - o))
        grid = torch.from_numpy(rng.standard_normal((cells, cells)).astype(np.float32)).to(device)
        acc += F.interpolate(grid[None, None], size=(size, size), mode="bilinear",
                             align_corners=False)[0, 0]
        del grid
    sd = float(acc.std())
    n_rect = n_prims // 2
    for _ in range(n_rect):
        hgt = int(rng.integers(8, 257)); wid = int(rng.integers(8, 257))
        y = int(rng.integers(0, size)); x = int(rng.integers(0, size))
        amp = float(rng.uniform(-3.0, 3.0)) * sd
        acc[y:min(size, y + hgt), x:min(size, x + wid)] += amp
    for _ in range(n_prims - n_rect):
        length = float(rng.integers(32, 513)); width = float(rng.integers(1, 4))
        ang = float(rng.uniform(0.0, np.pi))
        y0 = float(rng.uniform(0, size)); x0 = float(rng.uniform(0, size))
        y1 = y0 + length * np.sin(ang); x1 = x0 + length * np.cos(ang)
        amp = float(rng.uniform(-3.0, 3.0)) * sd
        r = width / 2.0 + 1.0
        ymin = int(max(0, np.floor(min(y0, y1) - r))); ymax = int(min(size, np.ceil(max(y0, y1) + r) + 1))
        xmin = int(max(0, np.floor(min(x0, x1) - r))); xmax = int(min(size, np.ceil(max(x0, x1) + r) + 1))
        if ymin >= ymax or xmin >= xmax:
            continue
        yy = torch.arange(ymin, ymax, dtype=torch.float32, device=device)[:, None]
        xx = torch.arange(xmin, xmax, dtype=torch.float32, device=device)[None, :]
        dy, dx = y1 - y0, x1 - x0
        tpar = (((yy - y0) * dy + (xx - x0) * dx) / max(dy * dy + dx * dx, 1e-12)).clamp(0.0, 1.0)
        d2 = (yy - (y0 + tpar * dy)) ** 2 + (xx - (x0 + tpar * dx)) ** 2
        acc[ymin:ymax, xmin:xmax] += (d2 <= (width / 2.0) ** 2).to(torch.float32) * amp
    lo, hi = float(acc.min()), float(acc.max())
    if hi <= lo:
        return torch.zeros((size, size), dtype=torch.uint8, device=device)
    acc -= lo
    acc *= 255.0 / (hi - lo)
    return torch.round(acc).to(torch.uint8)


# The serving workload: four resident images of the same generator (area-
# scaled primitives, one octave more per doubling of the side), seeds
# 2005..2008.
SERVE_IMAGES = {4096: dict(n_octaves=9, n_prims=800, seed=2005),
                8192: dict(n_octaves=10, n_prims=3200, seed=2006),
                12288: dict(n_octaves=10, n_prims=7200, seed=2007),
                16384: dict(n_octaves=11, n_prims=12800, seed=2008)}


def serve_image(size: int, device="cuda"):
    """One image of the serving workload, drawn on the device (uint8)."""
    return aerial_image_device(size, device=device, **SERVE_IMAGES[size])


def make_templates(img: np.ndarray, sizes, seed: int, noise: float,
                   gain=(0.8, 1.2), offset=(-20.0, 20.0), quantize: bool = False) -> list:
    """Crops at seeded top-left locations, a*x+b, plus N(0, noise^2). float32.

    quantize: round to integers and clip to 0..255, as an 8-bit camera would
    record the template (the paper's templates are images of the scene taken
    from another view point at another time); the values stay float32."""
    rng = np.random.default_rng(seed)
    p, q = img.shape
    out = []
    for s in sizes:
        m, n = (s, s) if np.isscalar(s) else s
        y = int(rng.integers(0, p - m + 1)); x = int(rng.integers(0, q - n + 1))
        a = float(rng.uniform(*gain)); b = float(rng.uniform(*offset))
        crop = np.asarray(img[y:y + m, x:x + n], dtype=np.float64)
        t = a * crop + b + rng.normal(0.0, noise, size=(m, n))
        if quantize:
            t = np.clip(np.rint(t), 0.0, 255.0)
        out.append(Template(np.ascontiguousarray(t.astype(np.float32)), y, x, a, b, noise))
    return out


# ---------------------------------------------------------------------------
# The workloads, by image and template sizes.  "image" recipes are (kind,
# kwargs); "templates" give the template sizes, seed and noise.
# ---------------------------------------------------------------------------
WORKLOADS = {
    "white256_16": dict(image=("white_blur", dict(size=256, seed=1001)),
            templates=dict(sizes=[16], seed=1101, noise=5.0, quantize=True),
            group=3, blur=False),
    "aerial2048_32and64": dict(image=("aerial", dict(size=2048, n_octaves=8, n_prims=200, seed=2002)),
            templates=dict(sizes=[32] * 8 + [64] * 8, seed=2102, noise=3.0, quantize=True),
            group=0, blur=True),
    "aerial8192_128": dict(image=("aerial", dict(size=8192, n_octaves=12, n_prims=3200, seed=2003)),
            templates=dict(sizes=[128] * 16, seed=2103, noise=3.0, quantize=True),
            group=0, blur=True),
    "aerial4096_batch256": dict(image=("aerial", dict(size=4096, n_octaves=9, n_prims=800, seed=2004)),
            templates=dict(sizes=None, seed=2104, noise=3.0, count=256, quantize=True),
            group=0, blur=True),
}


def workload_image(k: str) -> np.ndarray:
    kind, kw = WORKLOADS[k]["image"]
    if kind == "white_blur":
        return white_blur_image(**kw)
    return aerial_image(**kw)


def batch_sizes(count: int, seed: int) -> list:
    """Template sizes drawn uniformly from BATCH_SIZES (seeded)."""
    rng = np.random.default_rng(seed + 7)
    return [int(BATCH_SIZES[i]) for i in rng.integers(0, len(BATCH_SIZES), size=count)]


def workload_templates(k: str, img: np.ndarray, count: int | None = None) -> list:
    tc = WORKLOADS[k]["templates"]
    sizes = tc["sizes"]
    if sizes is None:
        sizes = batch_sizes(tc["count"], tc["seed"])
    if count is not None:
        sizes = sizes[:count]
    return make_templates(img, sizes, tc["seed"], tc["noise"], quantize=tc.get("quantize", False))
