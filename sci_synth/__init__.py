"""Seeded synthetic inputs for video snapshot compressive imaging (SCI).

This module draws the random inputs that both the FP64 oracle and the CUDA
path consume: ground-truth videos, binary modulation masks and measurement
noise.  It holds none of the reconstruction arithmetic (no forward operator,
no projection, no TV): it only produces arrays.

Layout convention: every video-shaped array is ``[B][nx][ny]`` (frame-major,
row-major), with ``i < nx`` the vertical (row) index and ``j < ny`` the
horizontal (column) index.  A measurement model after Eq. (3) of the paper
combines these arrays as ``Y = sum_k X_k * C_k + G``; that sum is computed by
the caller, not here.

Stand-in for the paper's data (Sec. 3): the Kobe/Traffic/Runner/Drop videos
(B = 8) and the 512x512x10 real hand measurement are not available, so the
videos here are textured ellipses translating over linear ramps, with the
shapes and frame counts of those workloads.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "Case", "CONFIGS", "video", "masks_bernoulli", "masks_shifted", "noise",
    "make_case", "pack_mask_bits", "batch_sizes", "masks_and_noise_torch",
]


def _rng(seed_or_rng) -> np.random.Generator:
    if isinstance(seed_or_rng, np.random.Generator):
        return seed_or_rng
    return np.random.default_rng(seed_or_rng)


def video(nx: int, ny: int, B: int, rng) -> np.ndarray:
    """A ``[B][nx][ny]`` float64 video in [0, 1].

    Background: linear ramp ``a*i/nx + b*j/ny`` with ``a, b ~ U[0, 0.3]``.
    Objects: 4 ellipses with semi-axes ``~ U[n/16, n/5]`` (n = min(nx, ny)),
    random orientation, sinusoidal texture
    ``0.5 + 0.25*sin(2*pi*(fx*i + fy*j) + phi)`` with ``f ~ U[1/32, 1/8]``
    cycles/pixel mapped into [0.3, 1], each translating by an integer velocity
    whose components are drawn from {+-1, +-2, +-3} pixels per frame.
    """
    rng = _rng(rng)
    n = min(nx, ny)
    a, b = rng.uniform(0.0, 0.3, size=2)
    ii = np.arange(nx, dtype=np.float64)[:, None]
    jj = np.arange(ny, dtype=np.float64)[None, :]
    base = a * ii / nx + b * jj / ny
    out = np.repeat(base[None, :, :], B, axis=0).copy()
    for _ in range(4):
        ra, rb = rng.uniform(n / 16.0, n / 5.0, size=2)
        ang = rng.uniform(0.0, np.pi)
        ci, cj = rng.uniform(0.2 * nx, 0.8 * nx), rng.uniform(0.2 * ny, 0.8 * ny)
        fx, fy = rng.uniform(1.0 / 32.0, 1.0 / 8.0, size=2)
        phi = rng.uniform(0.0, 2.0 * np.pi)
        vel = rng.choice(np.array([-3, -2, -1, 1, 2, 3]), size=2)
        ca, sa = np.cos(ang), np.sin(ang)
        tex = 0.5 + 0.25 * np.sin(2.0 * np.pi * (fx * ii + fy * jj) + phi)
        tex = 0.3 + 0.7 * (tex - 0.25) / 0.5  # [0.25, 0.75] -> [0.3, 1.0]
        reach = max(ra, rb) + 2.0
        for k in range(B):
            c0, c1 = ci + vel[0] * k, cj + vel[1] * k
            i0, i1 = max(0, int(np.floor(c0 - reach))), min(nx, int(np.ceil(c0 + reach)) + 1)
            j0, j1 = max(0, int(np.floor(c1 - reach))), min(ny, int(np.ceil(c1 + reach)) + 1)
            if i0 >= i1 or j0 >= j1:
                continue
            di = ii[i0:i1] - c0
            dj = jj[:, j0:j1] - c1
            u = (ca * di + sa * dj) / ra
            v = (-sa * di + ca * dj) / rb
            inside = (u * u + v * v) <= 1.0
            blk = out[k, i0:i1, j0:j1]
            out[k, i0:i1, j0:j1] = np.where(inside, tex[i0:i1, j0:j1], blk)
    return np.clip(out, 0.0, 1.0)


def masks_bernoulli(nx: int, ny: int, B: int, rng, p: float = 0.5) -> np.ndarray:
    """``B`` i.i.d. Bernoulli(p) binary masks, ``[B][nx][ny]`` uint8 in {0, 1}."""
    rng = _rng(rng)
    return (rng.random((B, nx, ny)) < p).astype(np.uint8)


def masks_shifted(nx: int, ny: int, B: int, rng, p: float = 0.5) -> np.ndarray:
    """One tall Bernoulli(p) mask of ``(nx + B - 1) x ny`` shifted 1 px per frame.

    Frame k sees rows ``[k, k + nx)`` of the tall mask: a mask translating
    vertically by one pixel per frame, with no wrap-around (the CACTI-style
    translating code the paper's introduction describes).
    """
    rng = _rng(rng)
    tall = (rng.random((nx + B - 1, ny)) < p).astype(np.uint8)
    return np.stack([tall[k:k + nx] for k in range(B)], axis=0)


def noise(nx: int, ny: int, sigma: float, rng) -> np.ndarray:
    """I.i.d. Gaussian measurement noise ``N(0, sigma^2)``, ``[nx][ny]`` float64."""
    rng = _rng(rng)
    if sigma == 0.0:
        return np.zeros((nx, ny))
    return rng.normal(0.0, sigma, size=(nx, ny))


def pack_mask_bits(masks: np.ndarray) -> np.ndarray:
    """Pack binary ``[B][nx][ny]`` masks into ``[nx][ny]`` uint32 words.

    Bit k of word (i, j) is mask k at pixel (i, j); B must be at most 32.
    This is a storage format only (no arithmetic of the method).
    """
    B = masks.shape[0]
    if B > 32:
        raise ValueError("at most 32 frames fit in one 32-bit mask word")
    if not np.all((masks == 0) | (masks == 1)):
        raise ValueError("masks must be binary (0 or 1)")
    words = np.zeros(masks.shape[1:], dtype=np.uint64)
    for k in range(B):
        words |= masks[k].astype(np.uint64) << np.uint64(k)
    return words.astype(np.uint32)


def batch_sizes(count: int, sizes, seed: int):
    """Sizes of `count` measurements drawn uniformly (seeded) from `sizes`."""
    rng = np.random.default_rng(np.random.SeedSequence(seed).spawn(4)[3])
    return [tuple(sizes[i]) for i in rng.integers(0, len(sizes), size=count)]


def masks_and_noise_torch(nx: int, ny: int, B: int, sigma: float, seed: int, device):
    """Bernoulli(0.5) masks (uint8 [B][nx][ny]) and N(0, sigma^2) noise
    ([nx][ny] float32) drawn on `device` from a seeded torch generator, for
    workloads too large to draw on the host."""
    import torch
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    m = (torch.rand((B, nx, ny), generator=gen, device=device) < 0.5).to(torch.uint8)
    g = torch.randn((nx, ny), generator=gen, device=device) * sigma
    return m, g


@dataclasses.dataclass(frozen=True)
class Case:
    """One synthetic SCI problem: ground truth, masks and noise (no measurement)."""
    x_gt: np.ndarray      # [B][nx][ny] float64 in [0, 1]
    masks: np.ndarray     # [B][nx][ny] uint8 in {0, 1}
    noise: np.ndarray     # [nx][ny] float64
    seed: int

    @property
    def shape(self):
        return self.x_gt.shape


def make_case(nx: int, ny: int, B: int, seed: int, *, mask: str = "bernoulli",
              sigma: float = 0.0) -> Case:
    """Draw a case from independent child streams of ``SeedSequence(seed)``.

    Streams: 0 = video, 1 = masks, 2 = noise, so changing one of them never
    shifts the others.
    """
    ss_video, ss_mask, ss_noise = np.random.SeedSequence(seed).spawn(3)
    x = video(nx, ny, B, np.random.default_rng(ss_video))
    if mask == "bernoulli":
        m = masks_bernoulli(nx, ny, B, np.random.default_rng(ss_mask))
    elif mask == "shifted":
        m = masks_shifted(nx, ny, B, np.random.default_rng(ss_mask))
    else:
        raise ValueError(f"unknown mask kind {mask!r}")
    g = noise(nx, ny, sigma, np.random.default_rng(ss_noise))
    return Case(x_gt=x, masks=m, noise=g, seed=seed)


# Workload shapes (sizes, iteration counts, mask kind, noise) of the five
# reconstruction settings this library is measured on.  lambda = 0.05 on data
# in [0, 1] throughout (the paper does not state lambda or the data scale).
CONFIGS = {
    "gap_atv_256x256x8": dict(nx=256, ny=256, B=8, seed=1, mask="bernoulli", sigma=0.0,
                              outer=50, inner=5, lam=0.05, tv=("atv",), algo=("gap",)),
    "sci_512x512x10": dict(nx=512, ny=512, B=10, seed=2, mask="shifted", sigma=0.01,
                           outer=200, inner=10, lam=0.05, rho=0.01,
                           tv=("atv", "itv2d", "vtv"), algo=("gap", "admm")),
    "gap_itv2d_2048x2048x32": dict(nx=2048, ny=2048, B=32, seed=3, mask="bernoulli",
                                   sigma=0.0, outer=100, inner=10, lam=0.05,
                                   tv=("itv2d",), algo=("gap",)),
    "batched_vtv_256": dict(count=256, sizes=((128, 128, 8), (256, 256, 8), (512, 512, 10),
                                              (1024, 1024, 24)),
                            seed=4, mask="bernoulli", sigma=0.01, outer=100, inner=5,
                            lam=0.05, tv=("vtv",), algo=("gap",)),
}
