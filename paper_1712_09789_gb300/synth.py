"""Seeded synthetic binary images shaped like the paper's workloads.

This module only draws inputs.  It holds none of the labelling arithmetic and
is shared, unchanged, by the tests, the benchmark and the CPU oracle checks,
so both sides of every comparison see the same bytes.

All images are ``uint8`` arrays of 0/1 (row-major, ``[H][W]``).  Random draws
use ``numpy.random.Generator(PCG64(seed))``.

Workload shapes (Sec. 4.1 evaluates square random-noise images from 32x32 to
4096x4096 at densities 0.1..0.9; Sec. 4.3 times 2048x2048 noise images and
natural/texture/artifact images from 512x512 to 4096x4096):

* ``bernoulli``      i.i.d. foreground with probability ``p``.
* ``granular``       one Bernoulli draw per ``g x g`` block (``g=1`` is plain noise).
* ``spiral``         one 1-px square spiral with 1-px gaps (a single component
                     that crosses every tile).
* ``rings``          concentric 1-px square rings, Chebyshev radius 0, 3, 6, ...
* ``comb``           serpentine comb: 1-px teeth every 2 columns, joined
                     alternately at the top and bottom row (one component).
* ``smoothed``       Gaussian-smoothed white noise thresholded at a quantile.
* ``batch_uneven``   256 images of uneven size for the batched path.
* ``serving_frames`` a stream of translated smoothed-noise frames.
* ``bernoulli3d``, ``smoothed3d``, ``shells``, ``comb3d``: volumes
  ``[D][H][W]`` for the 3D extension (noise, blobs, concentric cube shells,
  a comb per slice joined through the slices between them).
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def bernoulli(H: int, W: int, p: float, seed: int) -> np.ndarray:
    """I.i.d. foreground with probability ``p``."""
    return (rng(seed).random((H, W)) < p).astype(np.uint8)


def granular(H: int, W: int, p: float, g: int, seed: int) -> np.ndarray:
    """Each ``g x g`` block takes one Bernoulli(p) draw (ragged blocks cropped)."""
    bh, bw = -(-H // g), -(-W // g)
    blocks = (rng(seed).random((bh, bw)) < p).astype(np.uint8)
    return np.ascontiguousarray(np.repeat(np.repeat(blocks, g, axis=0), g, axis=1)[:H, :W])


def spiral(N: int) -> np.ndarray:
    """A 1-px square spiral with 1-px gaps filling an ``N x N`` image.

    Square rings sit at offsets k = 0, 2, 4, ...; each ring except the last is
    opened at pixel (x=k, y=k+1) and joined to the next ring by a bridge pixel
    at (x=k+1, y=k+2).  The result is one path, hence one component under both
    connectivities.
    """
    img = np.zeros((N, N), dtype=np.uint8)
    ks = list(range(0, (N - 1) // 2 + 1, 2))
    for i, k in enumerate(ks):
        lo, hi = k, N - 1 - k
        img[lo, lo:hi + 1] = 1
        img[hi, lo:hi + 1] = 1
        img[lo:hi + 1, lo] = 1
        img[lo:hi + 1, hi] = 1
        if i + 1 < len(ks):
            img[lo + 1, lo] = 0
            img[lo + 2, lo + 1] = 1
    return img


def rings(N: int) -> np.ndarray:
    """Concentric 1-px square rings around pixel (N//2, N//2).

    A ring of Chebyshev radius d (d = 0, 3, 6, ...) is drawn only if it lies
    entirely inside the image, so the image holds ``R_max // 3 + 1`` rings with
    ``R_max = min(N//2, N - 1 - N//2)``; radius 0 is the single centre pixel.
    """
    c = N // 2
    rmax = min(c, N - 1 - c)
    ys, xs = np.ogrid[:N, :N]
    d = np.maximum(np.abs(xs - c), np.abs(ys - c))
    return ((d % 3 == 0) & (d <= rmax - rmax % 3)).astype(np.uint8)


def ring_count(N: int) -> int:
    c = N // 2
    return min(c, N - 1 - c) // 3 + 1


def comb(H: int, W: int) -> np.ndarray:
    """Serpentine comb: full-height teeth on even columns; the gap between
    teeth 2i and 2i+2 is bridged in row 0 when i is even and in row H-1 when
    i is odd.  One component under both connectivities."""
    img = np.zeros((H, W), dtype=np.uint8)
    img[:, 0::2] = 1
    gaps = np.arange(1, W - 1, 2)
    top = gaps[(gaps // 2) % 2 == 0]
    bot = gaps[(gaps // 2) % 2 == 1]
    img[0, top] = 1
    img[H - 1, bot] = 1
    return img


def _gauss_smooth(field: np.ndarray, sigma: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter1d

    out = gaussian_filter1d(field, sigma, axis=0, mode="wrap")
    return gaussian_filter1d(out, sigma, axis=1, mode="wrap")


def smoothed_field(H: int, W: int, sigma: float, seed: int) -> np.ndarray:
    """Float64 white noise smoothed by a separable Gaussian (periodic edges)."""
    return _gauss_smooth(rng(seed).standard_normal((H, W)), sigma)


def smoothed(H: int, W: int, sigma: float, density: float, seed: int) -> np.ndarray:
    """Smoothed noise thresholded so that about ``density`` of it is foreground
    (``density=0.5`` thresholds at the median)."""
    f = smoothed_field(H, W, sigma, seed)
    t = np.quantile(f, 1.0 - density)
    return (f > t).astype(np.uint8)


# --- composite workloads --------------------------------------------------

def noise_4096_set(size: int = 4096, seeds=(0, 1, 2)):
    """The 4096x4096 single-image set: Bernoulli densities 0.1..0.9 and
    granular noise (g = 4, 16; g = 1 is the Bernoulli 0.5 image) at 0.5.
    Yields ``(name, image)``."""
    for s in seeds:
        for k in range(1, 10):
            p = k / 10
            yield f"bernoulli_p{p:.1f}_s{s}", bernoulli(size, size, p, s)
        for g in (4, 16):
            yield f"granular_g{g}_s{s}", granular(size, size, 0.5, g, s)


def stress_8192_set(size: int = 8192, seed: int = 0):
    """The 8192x8192 structured stress set.  Yields ``(name, image)``."""
    yield "spiral", spiral(size)
    yield "rings", rings(size)
    yield "comb", comb(size, size)
    yield "smoothed_sigma8", smoothed(size, size, 8.0, 0.5, seed)
    yield "bernoulli_p0.5", bernoulli(size, size, 0.5, seed)


def batch_uneven(n: int = 256, lo: int = 64, hi: int = 2048, seed: int = 0):
    """``n`` images with H, W uniform integers in [lo, hi] and density uniform
    in [0.2, 0.8]; the first half i.i.d. Bernoulli, the second half sigma=4
    smoothed noise thresholded at the (1 - density) quantile."""
    g = rng(seed)
    shapes = g.integers(lo, hi + 1, size=(n, 2))
    dens = g.uniform(0.2, 0.8, size=n)
    seeds = g.integers(0, 2**31 - 1, size=n)
    out = []
    for i in range(n):
        H, W = int(shapes[i, 0]), int(shapes[i, 1])
        if i < n // 2:
            out.append(bernoulli(H, W, float(dens[i]), int(seeds[i])))
        else:
            out.append(smoothed(H, W, 4.0, float(dens[i]), int(seeds[i])))
    return out


SERVING_SIZES = ((480, 640), (1080, 1920), (2160, 3840))
SERVING_MIX = (0.50, 0.35, 0.15)


def serving_frames(n_frames: int, n_streams: int = 4, seed: int = 0):
    """Frames for the serving stream: each request picks a size from the mix
    (640x480 50%, 1920x1080 35%, 3840x2160 15%) and a stream; each stream
    keeps one sigma=6 smoothed field per size with density in [0.3, 0.6] and
    translates it by 1-4 px per frame.  Returns a list of uint8 images."""
    g = rng(seed)
    size_idx = g.choice(len(SERVING_SIZES), size=n_frames, p=SERVING_MIX)
    stream_of = g.integers(0, n_streams, size=n_frames)
    fields = {}
    frames = []
    for i in range(n_frames):
        key = (int(stream_of[i]), int(size_idx[i]))
        H, W = SERVING_SIZES[key[1]]
        if key not in fields:
            d = float(g.uniform(0.3, 0.6))
            f = smoothed_field(H, W, 6.0, int(g.integers(0, 2**31 - 1)))
            fields[key] = [f, float(np.quantile(f, 1.0 - d))]
        f, t = fields[key]
        dy, dx = (int(v) for v in g.integers(1, 5, size=2))
        f = np.roll(f, (dy, dx), axis=(0, 1))
        fields[key][0] = f
        frames.append((f > t).astype(np.uint8))
    return frames


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process: exponential gaps."""
    g = rng(seed)
    n = int(rate_hz * duration_s * 1.2) + 16
    t = np.cumsum(g.exponential(1.0 / rate_hz, size=n))
    return t[t < duration_s]


# --- volumes ----------------------------------------------------------------
# 3D inputs are ``uint8`` arrays ``[D][H][W]`` (slice, row, column).

def bernoulli3d(D: int, H: int, W: int, p: float, seed: int) -> np.ndarray:
    """I.i.d. foreground voxels with probability ``p``; drawn slice by slice
    from one generator (the same stream as a single ``(D, H, W)`` draw)."""
    g = rng(seed)
    out = np.empty((D, H, W), dtype=np.uint8)
    for z in range(D):
        out[z] = g.random((H, W)) < p
    return out


def smoothed3d(D: int, H: int, W: int, sigma: float, density: float, seed: int) -> np.ndarray:
    """White noise smoothed by a separable Gaussian along all three axes
    (periodic edges), thresholded so that about ``density`` is foreground."""
    from scipy.ndimage import gaussian_filter1d

    f = rng(seed).standard_normal((D, H, W))
    for ax in range(3):
        f = gaussian_filter1d(f, sigma, axis=ax, mode="wrap")
    t = np.quantile(f, 1.0 - density)
    return (f > t).astype(np.uint8)


def shells(N: int) -> np.ndarray:
    """Concentric 1-voxel cube shells around voxel (N//2, N//2, N//2) at
    Chebyshev radius 0, 3, 6, ..., each drawn only if it lies inside the
    volume: ``ring_count(N)`` components under both connectivities."""
    c = N // 2
    rmax = min(c, N - 1 - c)
    zs, ys, xs = np.ogrid[:N, :N, :N]
    d = np.maximum(np.maximum(np.abs(xs - c), np.abs(ys - c)), np.abs(zs - c))
    return ((d % 3 == 0) & (d <= rmax - rmax % 3)).astype(np.uint8)


def comb3d(D: int, H: int, W: int) -> np.ndarray:
    """Even slices hold the serpentine ``comb(H, W)``; each odd slice holds the
    single voxel (x=0, y=0), which joins the combs above and below it.  One
    component under both connectivities, crossing every block face."""
    out = np.zeros((D, H, W), dtype=np.uint8)
    out[0::2] = comb(H, W)
    out[1::2, 0, 0] = 1
    return out
