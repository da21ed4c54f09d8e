"""Seeded synthetic binary images for labelling workloads.

This module only *makes inputs*. It holds none of the labelling arithmetic, so both
the CPU oracle tests and the CUDA path may draw their images from it.

The paper measures on USC-SIPI texture/aerial/misc images (1 MB or less) and on
binarised NLCD 2006 land-cover rasters (12 MB up to 465.20 MB), all binarised with
a 0.5 luminance threshold (Section V, Experiments; Table III).  Those datasets are
not available here, so the generators below stand in for them:

* ``bernoulli``      i.i.d. foreground with probability ``p`` (texture-like noise;
                     p sweeps across the 8-connected percolation threshold ~0.407).
* ``blobs``          Gaussian random field: white noise smoothed with a Gaussian of
                     ``sigma`` pixels (periodic boundary), thresholded at 0, giving
                     ~50% dense land-cover-like patches.
* ``serpentine``     a single 1-pixel-wide path that sweeps the whole image
                     (one component, longest possible union chains).
* closed-form patterns with known component counts (checkerboard, dot lattice,
  striped rows) used by the tests.

Every image is ``uint8`` with values {0, 1}, C-contiguous, shape (H, W).
"""
from __future__ import annotations

import hashlib
import math

import numpy as np

__all__ = [
    "bernoulli", "blobs", "serpentine", "checkerboard", "dot_lattice", "striped_rows",
    "batch_specs", "make_batch_image", "sha256", "sweep_8192", "pad_pitch", "blobs_device", "batch_device", "served_specs",
]


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def bernoulli(h: int, w: int, p: float, seed: int) -> np.ndarray:
    """I.i.d. Bernoulli(p) foreground: ``rng.random((h, w), float32) < p``."""
    rng = _rng(seed)
    return (rng.random((h, w), dtype=np.float32) < np.float32(p)).astype(np.uint8)


def _gauss_kernel(sigma: float) -> np.ndarray:
    r = int(math.ceil(4.0 * sigma))
    x = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-0.5 * (x / sigma) ** 2)
    return (k / k.sum()).astype(np.float32)


def _smooth_periodic(a: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian smoothing with wrap-around boundary (truncated at 4 sigma).

    Done as a circular convolution through the FFT along each axis, so large fields stay
    cheap; the result only feeds a threshold, and the thresholded bytes are what every
    consumer sees.
    """
    k = _gauss_kernel(sigma)
    r = (k.size - 1) // 2
    out = a
    for axis in (0, 1):
        n = out.shape[axis]
        kk = np.zeros(n, dtype=np.float32)
        for i, v in enumerate(k):
            kk[(i - r) % n] += v
        fk = np.fft.rfft(kk)
        fo = np.fft.rfft(out, axis=axis)
        shape = [1, 1]
        shape[axis] = fk.size
        out = np.fft.irfft(fo * fk.reshape(shape), n=n, axis=axis).astype(np.float32)
    return out


def blobs(h: int, w: int, sigma: float, seed: int, chunk_rows: int = 2048) -> np.ndarray:
    """Thresholded Gaussian random field: ``smooth_sigma(N(0,1) noise) > 0``.

    Large fields are built in row chunks for the first (row-axis) pass to bound memory.
    """
    rng = _rng(seed)
    noise = rng.standard_normal((h, w), dtype=np.float32)
    if h * w <= (1 << 26):
        f = _smooth_periodic(noise, sigma)
        return (f > 0).astype(np.uint8)
    # big images: smooth along columns (axis 1) chunk by chunk, then along rows (axis 0)
    k = _gauss_kernel(sigma)
    r = (k.size - 1) // 2
    kk = np.zeros(w, dtype=np.float32)
    for i, v in enumerate(k):
        kk[(i - r) % w] += v
    fk = np.fft.rfft(kk)
    for y0 in range(0, h, chunk_rows):
        y1 = min(h, y0 + chunk_rows)
        noise[y0:y1] = np.fft.irfft(np.fft.rfft(noise[y0:y1], axis=1) * fk[None, :], n=w, axis=1)
    kk = np.zeros(h, dtype=np.float32)
    for i, v in enumerate(k):
        kk[(i - r) % h] += v
    fk = np.fft.rfft(kk)
    out = np.empty((h, w), dtype=np.uint8)
    for x0 in range(0, w, chunk_rows):
        x1 = min(w, x0 + chunk_rows)
        col = np.fft.irfft(np.fft.rfft(noise[:, x0:x1], axis=0) * fk[:, None], n=h, axis=0)
        out[:, x0:x1] = col > 0
    return out


def _smooth_torch(noise, sigma: float):
    import torch

    device = noise.device
    k = _gauss_kernel(sigma)
    r = (k.size - 1) // 2
    for axis in (0, 1):
        n = noise.shape[axis]
        kk = np.zeros(n, dtype=np.float32)
        for i, v in enumerate(k):
            kk[(i - r) % n] += v
        fk = torch.fft.rfft(torch.from_numpy(kk).to(device))
        shape = [1, 1]
        shape[axis] = fk.numel()
        noise = torch.fft.irfft(torch.fft.rfft(noise, dim=axis) * fk.reshape(shape), n=n, dim=axis)
    return noise


def batch_device(specs, device):
    """The images of ``batch_specs`` as uint8 torch tensors on ``device`` (same recipe as
    ``make_batch_image``: Bernoulli items drawn on the host; blob items from host noise,
    smoothed and thresholded at their (1-p)-quantile on the device)."""
    import torch

    out = []
    for spec in specs:
        h, w = spec["h"], spec["w"]
        if spec["kind"] == "bernoulli":
            out.append(torch.from_numpy(bernoulli(h, w, spec["p"], spec["seed"])).to(device))
        else:
            rng = _rng(spec["seed"])
            noise = torch.from_numpy(rng.standard_normal((h, w), dtype=np.float32)).to(device)
            f = _smooth_torch(noise, spec["sigma"])
            v = f.reshape(-1)
            k = int(round((1.0 - spec["p"]) * (v.numel() - 1)))
            thr = torch.sort(v).values[k]
            out.append((f > thr).to(torch.uint8))
    return out


def blobs_device(h: int, w: int, sigma: float, seed: int, device):
    """Same recipe as ``blobs`` (numpy PCG64 noise, periodic Gaussian smoothing truncated at
    4 sigma, threshold at 0), with the smoothing done by torch FFTs on ``device``.  Returns a
    uint8 torch tensor on ``device``; callers that need the bytes on the host copy them, so
    every consumer still sees identical bytes."""
    import torch

    rng = _rng(seed)
    noise = torch.from_numpy(rng.standard_normal((h, w), dtype=np.float32)).to(device)
    k = _gauss_kernel(sigma)
    r = (k.size - 1) // 2
    for axis in (0, 1):
        n = noise.shape[axis]
        kk = np.zeros(n, dtype=np.float32)
        for i, v in enumerate(k):
            kk[(i - r) % n] += v
        fk = torch.fft.rfft(torch.from_numpy(kk).to(device))
        shape = [1, 1]
        shape[axis] = fk.numel()
        noise = torch.fft.irfft(torch.fft.rfft(noise, dim=axis) * fk.reshape(shape), n=n, dim=axis)
    return (noise > 0).to(torch.uint8)


def gray_field_device(h: int, w: int, sigma: float, seed: int, device):
    """8-bit grayscale stand-in for the paper's land-cover rasters before binarisation: the
    smoothed field of ``blobs_device`` scaled to unit variance and quantised as
    clip(round(128 + 40 z), 0, 255).  Thresholding at 127 keeps z > -0.0125, about half the
    pixels, near the percolation point of the field."""
    import torch

    rng = _rng(seed)
    noise = torch.from_numpy(rng.standard_normal((h, w), dtype=np.float32)).to(device)
    k = _gauss_kernel(sigma)
    r = (k.size - 1) // 2
    for axis in (0, 1):
        n = noise.shape[axis]
        kk = np.zeros(n, dtype=np.float32)
        for i, v in enumerate(k):
            kk[(i - r) % n] += v
        fk = torch.fft.rfft(torch.from_numpy(kk).to(device))
        shape = [1, 1]
        shape[axis] = fk.numel()
        noise = torch.fft.irfft(torch.fft.rfft(noise, dim=axis) * fk.reshape(shape), n=n, dim=axis)
    z = noise / noise.std()
    return torch.clamp(torch.round(128.0 + 40.0 * z), 0, 255).to(torch.uint8)


def classes_device(h: int, w: int, sigma: float, ncls: int, seed: int, device, background: float = 0.1):
    """Multi-class stand-in for a land-cover raster: a smoothed Gaussian field (as in
    ``blobs_device``) cut at its equal-mass quantiles into classes 1..ncls, and byte 0 (no
    data) where an independent smoothed field lies below its ``background`` quantile."""
    import torch

    def field(sd):
        rng = _rng(sd)
        noise = torch.from_numpy(rng.standard_normal((h, w), dtype=np.float32)).to(device)
        k = _gauss_kernel(sigma)
        r = (k.size - 1) // 2
        for axis in (0, 1):
            n = noise.shape[axis]
            kk = np.zeros(n, dtype=np.float32)
            for i, v in enumerate(k):
                kk[(i - r) % n] += v
            fk = torch.fft.rfft(torch.from_numpy(kk).to(device))
            shape = [1, 1]
            shape[axis] = fk.numel()
            noise = torch.fft.irfft(torch.fft.rfft(noise, dim=axis) * fk.reshape(shape), n=n, dim=axis)
        return noise.reshape(-1)

    f = field(seed)
    srt = torch.sort(f).values
    m = f.numel()
    cuts = torch.stack([srt[min(m - 1, (m * j) // ncls)] for j in range(1, ncls)]) if ncls > 1 else srt[:0]
    cls = (torch.bucketize(f, cuts, right=True) + 1).to(torch.uint8)
    if background > 0:
        g = field(seed + 7919)
        thr = torch.sort(g).values[int(background * (m - 1))]
        cls[g < thr] = 0
    return cls.reshape(h, w)


def serpentine(h: int, w: int) -> np.ndarray:
    """One 1-px-wide path covering the image: even rows full; odd row y holds a single
    pixel at x = W-1 when y % 4 == 1 and at x = 0 when y % 4 == 3.  One component
    under 8- and 4-connectivity."""
    img = np.zeros((h, w), dtype=np.uint8)
    img[0::2, :] = 1
    img[1::4, w - 1] = 1
    img[3::4, 0] = 1
    return img


def checkerboard(h: int, w: int, phase: int = 0) -> np.ndarray:
    y, x = np.indices((h, w))
    return (((y + x + phase) & 1) == 0).astype(np.uint8)


def dot_lattice(h: int, w: int) -> np.ndarray:
    """Pixels at (2i, 2j): ceil(H/2)*ceil(W/2) isolated components."""
    img = np.zeros((h, w), dtype=np.uint8)
    img[0::2, 0::2] = 1
    return img


def striped_rows(h: int, w: int) -> np.ndarray:
    """Full rows at even y: ceil(H/2) components."""
    img = np.zeros((h, w), dtype=np.uint8)
    img[0::2, :] = 1
    return img


def sha256(img: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(img).tobytes()).hexdigest()


def pad_pitch(img: np.ndarray, pitch: int, fill: int = 7) -> np.ndarray:
    """Copy ``img`` into rows of ``pitch`` bytes; the padding bytes hold ``fill`` so that
    a reader that wrongly looks past column W-1 sees foreground."""
    h, w = img.shape
    assert pitch >= w
    out = np.full((h, pitch), fill, dtype=np.uint8)
    out[:, :w] = img
    return out


# ---- workload recipes -------------------------------------------------------------

SWEEP_8192 = [("bernoulli", 0.1, 2), ("bernoulli", 0.3, 3), ("bernoulli", 0.5, 4),
              ("bernoulli", 0.7, 5), ("bernoulli", 0.9, 6), ("blobs", 4.0, 7)]


def sweep_8192(side: int = 8192):
    """The 8192x8192 density sweep: Bernoulli p in {0.1,0.3,0.5,0.7,0.9} (seeds 2..6)
    plus a sigma=4 thresholded field (seed 7).  Yields (name, image)."""
    for kind, arg, seed in SWEEP_8192:
        if kind == "bernoulli":
            yield f"bernoulli_p{arg}", bernoulli(side, side, arg, seed)
        else:
            yield f"blobs_sigma{arg:g}", blobs(side, side, arg, seed)


def batch_specs(n: int = 4096, seed: int = 100, lo: int = 64, hi: int = 2048):
    """Uneven batch recipe: H and W independently floor(exp(U(ln lo, ln hi))),
    density p ~ U(0.2, 0.8); even items Bernoulli(p), odd items blobs with sigma drawn
    from {2, 4, 8} (thresholded at the p-quantile so density ~= p)."""
    rng = _rng(seed)
    specs = []
    for i in range(n):
        h = int(math.floor(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        w = int(math.floor(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        p = float(rng.uniform(0.2, 0.8))
        sigma = float(rng.choice([2.0, 4.0, 8.0]))
        specs.append({"h": h, "w": w, "p": p, "kind": "bernoulli" if i % 2 == 0 else "blobs",
                      "sigma": sigma, "seed": seed * 100003 + i})
    return specs


def served_specs(n: int = 32, seed: int = 200, lo: int = 256, hi: int = 8192):
    """Request images for the serving workload: square, side floor(exp(U(ln lo, ln hi))),
    density p ~ U(0.2, 0.8), alternating Bernoulli(p) and sigma in {2,4,8} blobs."""
    rng = _rng(seed)
    specs = []
    for i in range(n):
        side = int(math.floor(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        specs.append({"h": side, "w": side, "p": float(rng.uniform(0.2, 0.8)),
                      "kind": "bernoulli" if i % 2 == 0 else "blobs",
                      "sigma": float(rng.choice([2.0, 4.0, 8.0])), "seed": seed * 100003 + i})
    return specs


def make_batch_image(spec) -> np.ndarray:
    h, w = spec["h"], spec["w"]
    if spec["kind"] == "bernoulli":
        return bernoulli(h, w, spec["p"], spec["seed"])
    rng = _rng(spec["seed"])
    noise = rng.standard_normal((h, w), dtype=np.float32)
    f = _smooth_periodic(noise, spec["sigma"])
    thr = np.quantile(f, 1.0 - spec["p"])
    return (f > thr).astype(np.uint8)
