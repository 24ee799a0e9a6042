"""Seeded synthetic fields shaped like the paper's workloads (Table 2).

The paper evaluates on SDRBench fields (CESM-ATM, HACC, HURR, Nyx) that are
not available here; these generators stand in for them with the same shapes
and a similar structure.  This module holds none of the compression method's
arithmetic: it only makes inputs, which both the CUDA path and the CPU oracle
then read byte for byte.

Every generator is deterministic for a given seed and device.  Large fields
are made with torch (on the GPU when one is present) in float64 and cast to
float32; small ones can be made on the CPU.
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _dev(device):
    if device is None:
        return torch.device("cuda" if torch.cuda.is_available() else "cpu")
    return torch.device(device)


# --------------------------------------------------------------------------
# 3D: Gaussian blobs + sinusoids + noise (the small 64^3 case)
# --------------------------------------------------------------------------
def blobs3d(shape=(64, 64, 64), seed: int = 1, n_blobs: int = 32, n_sin: int = 3, noise: float = 1e-3,
            device="cpu") -> torch.Tensor:
    """Sum of Gaussian blobs (centres uniform in the box, sigma U[2,8] cells,
    amplitude U[-1,1]) plus sinusoids (amplitude U[0.1,0.3], random unit
    direction, wavelength U[8,64] cells, random phase) plus N(0, noise).
    ``shape`` is (nz, ny, nx), C order, x fastest."""
    dev = _dev(device)
    g = _gen(seed, dev)
    nz, ny, nx = shape
    f64 = torch.float64
    z = torch.arange(nz, device=dev, dtype=f64).view(nz, 1, 1)
    y = torch.arange(ny, device=dev, dtype=f64).view(1, ny, 1)
    x = torch.arange(nx, device=dev, dtype=f64).view(1, 1, nx)
    out = torch.zeros(shape, device=dev, dtype=f64)
    ext = torch.tensor([nx, ny, nz], device=dev, dtype=f64)
    for _ in range(n_blobs):
        c = torch.rand(3, generator=g, device=dev, dtype=f64) * ext
        s = 2.0 + 6.0 * torch.rand(1, generator=g, device=dev, dtype=f64)
        a = 2.0 * torch.rand(1, generator=g, device=dev, dtype=f64) - 1.0
        r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
        out += a * torch.exp(-r2 / (2.0 * s * s))
    for _ in range(n_sin):
        a = 0.1 + 0.2 * torch.rand(1, generator=g, device=dev, dtype=f64)
        d = torch.randn(3, generator=g, device=dev, dtype=f64)
        d = d / d.norm()
        lam = 8.0 + 56.0 * torch.rand(1, generator=g, device=dev, dtype=f64)
        ph = 2.0 * math.pi * torch.rand(1, generator=g, device=dev, dtype=f64)
        out += a * torch.sin(2.0 * math.pi * (d[0] * x + d[1] * y + d[2] * z) / lam + ph)
    out += noise * torch.randn(shape, generator=g, device=dev, dtype=f64)
    return out.to(torch.float32)


# --------------------------------------------------------------------------
# 3D: Gaussian random field with a Kolmogorov spectrum (stands in for Nyx 512^3)
# --------------------------------------------------------------------------
def grf3d(n: int = 512, seed: int = 2, slope: float = 5.0 / 3.0, device=None) -> torch.Tensor:
    """Gaussian random field on an n^3 periodic grid whose shell-integrated
    energy spectrum falls as k^-slope (Kolmogorov for 5/3): white noise is
    transformed, each mode's amplitude is scaled by |k|^-(slope+2)/2, the k=0
    mode is removed, and the result is normalised to unit standard deviation."""
    dev = _dev(device)
    g = _gen(seed, dev)
    w = torch.randn((n, n, n), generator=g, device=dev, dtype=torch.float64)
    F = torch.fft.rfftn(w)
    del w
    k1 = torch.fft.fftfreq(n, d=1.0 / n, device=dev, dtype=torch.float64)
    kr = torch.fft.rfftfreq(n, d=1.0 / n, device=dev, dtype=torch.float64)
    k2 = k1.view(n, 1, 1) ** 2 + k1.view(1, n, 1) ** 2 + kr.view(1, 1, -1) ** 2
    k2[0, 0, 0] = 1.0
    F *= k2 ** (-(slope + 2.0) / 4.0)
    F[0, 0, 0] = 0.0
    del k2
    f = torch.fft.irfftn(F, s=(n, n, n))
    del F
    f /= f.std()
    return f.to(torch.float32)


# --------------------------------------------------------------------------
# 1D: clustered particle coordinates (stands in for HACC, 280,953,867 values)
# --------------------------------------------------------------------------
HACC_N = 280_953_867


def hacc1d(n: int = HACC_N, seed: int = 3, n_halos: int | None = None, device=None) -> torch.Tensor:
    """Coordinates in [0, 256): 80% of particles in Gaussian halos (sizes from
    a power law, sigma U[0.05, 1], wrapped periodically), 20% background in
    runs of ~1000 particles, each run uniform within its own slab of width
    U[0.5, 4] (as a rank's sub-domain in a particle dump).  Particles are
    emitted halo by halo, with halos and background runs in random order, so
    the series is locally clustered but unsorted."""
    dev = _dev(device)
    g = _gen(seed, dev)
    f64 = torch.float64
    if n_halos is None:
        n_halos = max(1, min(100_000, n // 2000))
    n_halo_p = int(round(0.8 * n))
    n_bg = n - n_halo_p
    # power-law (Pareto, index 1.5) halo sizes normalised to n_halo_p particles
    u = torch.rand(n_halos, generator=g, device=dev, dtype=f64).clamp_min(1e-12)
    w = u ** (-1.0 / 1.5)
    sizes = torch.floor(w / w.sum() * n_halo_p).to(torch.int64)
    short = n_halo_p - int(sizes.sum())
    if short > 0:
        idx = torch.randperm(n_halos, generator=g, device=dev)[:short] if short <= n_halos else None
        if idx is None:
            sizes += short // n_halos
            sizes[: short % n_halos] += 1
        else:
            sizes[idx] += 1
    # background in runs of ~1000 particles
    n_runs = max(1, n_bg // 1000)
    bsz = torch.full((n_runs,), n_bg // n_runs, dtype=torch.int64, device=dev)
    bsz[: n_bg % n_runs] += 1
    seg_sizes = torch.cat([sizes, bsz])
    n_seg = seg_sizes.numel()
    centre = 256.0 * torch.rand(n_halos + n_runs, generator=g, device=dev, dtype=f64)
    width = torch.cat([torch.zeros(n_halos, device=dev, dtype=f64),
                       0.5 + 3.5 * torch.rand(n_runs, generator=g, device=dev, dtype=f64)])
    sigma = torch.cat([0.05 + 0.95 * torch.rand(n_halos, generator=g, device=dev, dtype=f64),
                       torch.zeros(n_runs, device=dev, dtype=f64)])
    is_bg = torch.cat([torch.zeros(n_halos, dtype=torch.bool, device=dev),
                       torch.ones(n_runs, dtype=torch.bool, device=dev)])
    order = torch.randperm(n_seg, generator=g, device=dev)
    seg = torch.repeat_interleave(order, seg_sizes[order])
    out = torch.empty(n, dtype=torch.float32, device=dev)
    step = 1 << 26
    for s in range(0, n, step):
        e = min(n, s + step)
        sg = seg[s:e]
        r = torch.randn(e - s, generator=g, device=dev, dtype=f64)
        ub = width[sg] * torch.rand(e - s, generator=g, device=dev, dtype=f64)
        v = torch.where(is_bg[sg], centre[sg] + ub, centre[sg] + sigma[sg] * r)
        v = torch.remainder(v, 256.0)
        out[s:e] = v.to(torch.float32)
    return out


# --------------------------------------------------------------------------
# 2D: smooth lat/lon field from spherical harmonics (stands in for one CESM level)
# --------------------------------------------------------------------------
def cesm2d(ny: int = 1800, nx: int = 3600, seed: int = 4, lmax: int = 64, noise_rel: float = 1e-3) -> torch.Tensor:
    """sum_{l<=lmax} sum_m a_lm Y_lm on an ny x nx lat/lon grid with
    a_lm ~ N(0, (l+1)^-2), using orthonormal associated Legendre functions by
    the standard three-term recurrence in l for each m and an inverse real FFT
    over longitude; plus N(0, noise_rel * std) noise.  Computed on the CPU in
    float64 (numpy), returned as a float32 tensor of shape (ny, nx)."""
    rng = np.random.default_rng(seed)
    theta = (np.arange(ny) + 0.5) * np.pi / ny
    ct, st = np.cos(theta), np.sin(theta)
    coef = np.zeros((lmax + 1, lmax + 1), np.complex128)
    for l in range(lmax + 1):
        s = 1.0 / (l + 1)
        coef[l, 0] = s * rng.standard_normal()
        for m in range(1, l + 1):
            coef[l, m] = s * (rng.standard_normal() + 1j * rng.standard_normal()) / math.sqrt(2.0)
    spec = np.zeros((ny, nx // 2 + 1), np.complex128)
    pmm = np.full(ny, math.sqrt(1.0 / (4.0 * math.pi)))
    for m in range(lmax + 1):
        if m > 0:
            pmm = -math.sqrt((2.0 * m + 1.0) / (2.0 * m)) * st * pmm
        acc = coef[m, m] * pmm
        if m < lmax:
            p_lm2, p_lm1 = pmm, math.sqrt(2.0 * m + 3.0) * ct * pmm
            acc = acc + coef[m + 1, m] * p_lm1
            for l in range(m + 2, lmax + 1):
                a = math.sqrt((4.0 * l * l - 1.0) / (l * l - m * m))
                b = math.sqrt(((l - 1.0) ** 2 - m * m) / (4.0 * (l - 1.0) ** 2 - 1.0))
                p_l = a * (ct * p_lm1 - b * p_lm2)
                acc = acc + coef[l, m] * p_l
                p_lm2, p_lm1 = p_lm1, p_l
        spec[:, m] = acc * (nx if m == 0 else nx / 2.0)
    f = np.fft.irfft(spec, n=nx, axis=1)
    f = f + noise_rel * f.std() * rng.standard_normal(f.shape)
    return torch.from_numpy(f.astype(np.float32))


# --------------------------------------------------------------------------
# small helpers for tests
# --------------------------------------------------------------------------
def smooth_nd(shape, seed: int = 0) -> torch.Tensor:
    """Small smooth field of any shape (sum of a few separable sinusoids plus
    noise); used for ragged-shape cases in the tests."""
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[np.arange(s, dtype=np.float64) for s in shape], indexing="ij")
    f = np.zeros(shape, np.float64)
    for _ in range(4):
        ph = rng.uniform(0, 2 * np.pi)
        arg = sum(rng.uniform(0.02, 0.3) * gg for gg in grids) + ph
        f += rng.uniform(0.2, 1.0) * np.sin(arg)
    f += 1e-3 * rng.standard_normal(shape)
    return torch.from_numpy(f.astype(np.float32))


# --------------------------------------------------------------------------
# 3D: stitched field for the learned predictor selector
# --------------------------------------------------------------------------
def stitched3d(n: int = 512, seed: int = 200, region: int = 64, device=None) -> torch.Tensor:
    """n^3 field made of region^3 cubes, each (by seed) smooth (40%: Gaussian
    random field with a k^-4 spectrum), oscillatory (40%: a sinusoid with
    random direction, wavelength U[4,16] cells, amplitude 1, over a weak
    smooth background) or noisy (20%: uniform U[-a, a] with a U[0.05, 0.5]).
    Amplitudes are comparable so that one value-range bound fits all three."""
    dev = _dev(device)
    g = _gen(seed, dev)
    f64 = torch.float64
    smooth = grf3d(n, seed=seed * 7 + 1, slope=4.0 - 2.0, device=dev).to(f64)  # shell spectrum k^-2 -> P(k) ~ k^-4
    smooth = smooth / smooth.abs().max()
    nr = n // region
    out = torch.empty((n, n, n), dtype=f64, device=dev)
    ax = torch.arange(region, device=dev, dtype=f64)
    zz, yy, xx = torch.meshgrid(ax, ax, ax, indexing="ij")
    for rz in range(nr):
        for ry in range(nr):
            for rx in range(nr):
                sl = (slice(rz * region, (rz + 1) * region), slice(ry * region, (ry + 1) * region),
                      slice(rx * region, (rx + 1) * region))
                u = float(torch.rand(1, generator=g, device=dev, dtype=f64))
                base = smooth[sl]
                if u < 0.4:
                    out[sl] = base
                elif u < 0.8:
                    d = torch.randn(3, generator=g, device=dev, dtype=f64)
                    d = d / d.norm()
                    lam = 4.0 + 12.0 * float(torch.rand(1, generator=g, device=dev, dtype=f64))
                    ph = 2.0 * math.pi * float(torch.rand(1, generator=g, device=dev, dtype=f64))
                    out[sl] = torch.sin(2.0 * math.pi * (d[0] * (xx + rx * region) + d[1] * (yy + ry * region)
                                                         + d[2] * (zz + rz * region)) / lam + ph) + 0.1 * base
                else:
                    a = 0.05 + 0.45 * float(torch.rand(1, generator=g, device=dev, dtype=f64))
                    out[sl] = a * (2.0 * torch.rand(base.shape, generator=g, device=dev, dtype=f64) - 1.0)
    return out.to(torch.float32)


# --------------------------------------------------------------------------
# batched workload: many fields of uneven size
# --------------------------------------------------------------------------
def batch_fields(seed: int = 5, n3: int = 32, n2: int = 32, scale: float = 1.0, device=None):
    """n3 3D cubes with side U{32..256} (blob/sinusoid fields, blob count
    proportional to the volume: 32 per 64^3, between 8 and 512) and n2 2D
    lat/lon fields with each side U{512..4096} (spherical-harmonic fields),
    in a seeded random order.  ``scale`` shrinks every side (for tests).
    Returns a list of float32 tensors on ``device``."""
    rng = np.random.default_rng(seed)
    dev = _dev(device)
    specs = []
    for _ in range(n3):
        side = max(2, int(round(int(rng.integers(32, 257)) * scale)))
        specs.append(("3d", side, int(rng.integers(1 << 30))))
    for _ in range(n2):
        ny = max(8, int(round(int(rng.integers(512, 4097)) * scale)))
        nx = max(160, int(round(int(rng.integers(512, 4097)) * scale)))
        specs.append(("2d", (ny, nx), int(rng.integers(1 << 30))))
    order = rng.permutation(len(specs))
    out = []
    for i in order:
        kind, size, s = specs[i]
        if kind == "3d":
            nb = int(min(512, max(8, round(32 * size ** 3 / 64 ** 3))))
            out.append(blobs3d((size, size, size), seed=s, n_blobs=nb, device=dev).contiguous())
        else:
            out.append(cesm2d(size[0], size[1], seed=s).to(dev).contiguous())
    return out
