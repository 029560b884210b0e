"""Seeded synthetic scientific fields (stand-ins for the SDRBench fields of Table 2).

This module only *generates input data*; it contains none of the compressor's
arithmetic, so both the CUDA path and the CPU oracle can consume the same bytes.

The shapes follow Table 2 of the paper (HACC 1-D, CESM 1800x3600, Hurricane
100x500x500, Nyx 512^3); the value distributions are synthetic:

* ``walk_sines``: random walk with N(0,1) steps plus 8 sinusoids
  (frequencies log-uniform in [4/n, 0.05] cycles/sample, amplitudes U[1,100],
  phases U[0, 2pi)), a 1-D particle-like trace.
* ``grf``: Gaussian random field by spectral synthesis -- white noise, FFT,
  amplitude |k|^(-beta/2) for power spectrum |k|^-beta (k in cycles per domain,
  DC removed), inverse FFT, normalised to zero mean and unit variance.
* ``zero_patches`` / ``zero_blocks``: exact 0.0 regions (sparsity), either
  random 64x64 patches plus whole rows, or aligned cubes.

All generation runs on the given torch device with a seeded torch.Generator, so a
run is reproducible on one machine; CPU and CUDA generators produce different
streams, which is fine because every comparison feeds the same bytes to both
sides.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def walk_sines(n: int, seed: int, device="cpu") -> torch.Tensor:
    """1-D random walk (N(0,1) steps) plus a sum of 8 seeded sinusoids, FP32."""
    g = _gen(seed, device)
    steps = torch.randn(n, generator=g, device=device, dtype=torch.float64)
    walk = torch.cumsum(steps, 0)
    u = torch.rand(3, 8, generator=g, device=device, dtype=torch.float64)
    lo, hi = math.log(4.0 / max(n, 8)), math.log(0.05)
    freq = torch.exp(lo + (hi - lo) * u[0])
    amp = 1.0 + 99.0 * u[1]
    phase = 2.0 * math.pi * u[2]
    i = torch.arange(n, device=device, dtype=torch.float64)
    out = walk.clone()
    for k in range(8):
        out += amp[k] * torch.sin(2.0 * math.pi * freq[k] * i + phase[k])
    return out.to(torch.float32)


def grf(shape, beta: float, seed: int, device="cpu") -> torch.Tensor:
    """Gaussian random field with power spectrum |k|^-beta, unit variance, FP32."""
    shape = tuple(int(s) for s in shape)
    g = _gen(seed, device)
    noise = torch.randn(shape, generator=g, device=device, dtype=torch.float32)
    if torch.device(device).type == "cpu":
        # host fields go through numpy's FFT (double precision): some builds of torch's
        # CPU FFT corrupt memory on odd 3-D shapes
        return _grf_host(noise.numpy(), beta)
    spec = torch.fft.rfftn(noise)
    del noise
    k2 = None
    for ax, s in enumerate(shape):
        if ax == len(shape) - 1:
            f = torch.fft.rfftfreq(s, d=1.0 / s, device=device)
        else:
            f = torch.fft.fftfreq(s, d=1.0 / s, device=device)
        view = [1] * len(shape)
        view[ax] = -1
        f2 = (f.to(torch.float32) ** 2).view(view)
        k2 = f2 if k2 is None else k2 + f2
    amp = torch.where(k2 > 0, k2.clamp_min(1e-30) ** (-beta / 4.0), torch.zeros_like(k2))
    spec *= amp
    del amp, k2
    out = torch.fft.irfftn(spec, s=shape)
    del spec
    # cuFFT plans keep their own work areas outside PyTorch's allocator; fields of
    # many distinct shapes would otherwise pin tens of GB
    torch.backends.cuda.cufft_plan_cache[out.device.index].clear()
    out = out - out.mean()
    sd = out.std()
    if float(sd) > 0:
        out = out / sd
    return out.to(torch.float32).contiguous()


def _grf_host(noise: np.ndarray, beta: float) -> torch.Tensor:
    shape = noise.shape
    axes = list(range(len(shape)))
    spec = np.fft.rfftn(noise.astype(np.float64), axes=axes)
    k2 = np.zeros(spec.shape, dtype=np.float64)
    for ax, s in enumerate(shape):
        f = np.fft.rfftfreq(s, d=1.0 / s) if ax == len(shape) - 1 else np.fft.fftfreq(s, d=1.0 / s)
        view = [1] * len(shape)
        view[ax] = -1
        k2 = k2 + (f ** 2).reshape(view)
    amp = np.zeros_like(k2)
    pos = k2 > 0
    amp[pos] = k2[pos] ** (-beta / 4.0)
    out = np.fft.irfftn(spec * amp, s=shape, axes=axes)
    out = out - out.mean()
    sd = out.std()
    if sd > 0:
        out = out / sd
    return torch.from_numpy(np.ascontiguousarray(out.astype(np.float32)))


def zero_patches(x: torch.Tensor, frac: float, seed: int, patch: int = 64) -> torch.Tensor:
    """Set random patch x patch squares and whole rows of a 2-D field to exactly 0.0
    until at least `frac` of the cells are zero."""
    ny, nx = x.shape
    rng = np.random.default_rng(seed)
    mask = np.zeros((ny, nx), dtype=bool)
    target = int(math.ceil(frac * ny * nx))
    count = 0
    while count < target:
        if rng.random() < 0.25:
            r = int(rng.integers(0, ny))
            count += int((~mask[r]).sum())
            mask[r] = True
        else:
            y0 = int(rng.integers(0, max(1, ny - patch + 1)))
            x0 = int(rng.integers(0, max(1, nx - patch + 1)))
            sub = mask[y0:y0 + patch, x0:x0 + patch]
            count += int((~sub).sum())
            sub[...] = True
    m = torch.from_numpy(mask).to(x.device)
    return x.masked_fill(m, 0.0)


def zero_blocks(x: torch.Tensor, frac: float, seed: int, edge: int = 16) -> torch.Tensor:
    """Set randomly chosen aligned edge^ndim blocks to exactly 0.0 until at least
    `frac` of the cells are zero (1-, 2- or 3-D); some cells always stay non-zero."""
    shape = x.shape
    grid = [int(math.ceil(s / edge)) for s in shape]
    nb = int(np.prod(grid))
    rng = np.random.default_rng(seed)
    order = rng.permutation(nb)
    total = int(np.prod(shape))
    target = int(math.ceil(frac * total))
    cellmask = np.zeros(nb, dtype=bool)
    count = 0
    for b in order:
        if count >= target:
            break
        idx = np.unravel_index(int(b), grid)
        cells = 1
        for d, i in enumerate(idx):
            cells *= min(edge, shape[d] - i * edge)
        if count + cells >= total:
            continue  # never zero a whole field (its value range would be empty)
        cellmask[b] = True
        count += cells
    m = torch.from_numpy(cellmask.reshape(grid))
    for d in range(len(shape)):
        m = m.repeat_interleave(edge, dim=d)
    m = m[tuple(slice(0, s) for s in shape)].to(x.device)
    return x.masked_fill(m, 0.0)


@dataclass
class FieldSpec:
    """One synthetic workload: shape (slowest first), generator recipe, eb."""
    name: str
    dims: tuple
    eb_mode: str = "rel"
    eb: float = 1e-4
    recipe: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(np.prod(self.dims))


def make_field(spec: FieldSpec, device="cpu") -> torch.Tensor:
    r = spec.recipe
    kind = r.get("kind")
    seed = int(r.get("seed", 0))
    if kind == "walk_sines":
        x = walk_sines(spec.n, seed, device)
    elif kind == "grf":
        x = grf(spec.dims, float(r["beta"]), seed, device)
    elif kind == "lognormal":
        x = torch.exp(float(r.get("sigma", 1.5)) * grf(spec.dims, float(r["beta"]), seed, device))
    else:
        raise ValueError(f"unknown recipe {kind!r}")
    x = x.reshape(spec.dims)
    if r.get("zero_patches"):
        x = zero_patches(x, float(r["zero_patches"]), seed + 7919)
    if r.get("zero_blocks"):
        x = zero_blocks(x, float(r["zero_blocks"]), seed + 7919, int(r.get("zero_edge", 16)))
    return x.contiguous()


# The five workloads (shapes of Table 2; recipes as documented above).
def workload_1d(n: int = 1 << 20, seed: int = 1) -> FieldSpec:
    """1-D FP32 random walk plus 8 sines, rel eb 1e-3 (HACC-like trace)."""
    return FieldSpec("1d_walk_sines", (n,), "rel", 1e-3, {"kind": "walk_sines", "seed": seed})


def workload_2d(ny: int = 1800, nx: int = 3600, seed: int = 2) -> FieldSpec:
    """2-D 1800x3600 GRF k^-3 with 20% exact zeros (CESM-like), rel eb 1e-4."""
    return FieldSpec("2d_grf_k3_zero20", (ny, nx), "rel", 1e-4,
                     {"kind": "grf", "beta": 3.0, "seed": seed, "zero_patches": 0.20})


def workload_3d(n: int = 512, seed: int = 3, eb: float = 1e-4) -> FieldSpec:
    """3-D 512^3 log-normal density exp(1.5 g), g a GRF k^-2.5 (Nyx-like)."""
    return FieldSpec("3d_lognormal_k2.5", (n, n, n), "rel", eb,
                     {"kind": "lognormal", "beta": 2.5, "sigma": 1.5, "seed": seed})


def workload_selector(seed: int, dims=(100, 500, 500), eb: float = 1e-3) -> FieldSpec:
    """3-D 100x500x500 GRF k^-3 with aligned 16^3 zero blocks, zero fraction U[0,0.6]."""
    rng = np.random.default_rng(seed)
    frac = float(rng.uniform(0.0, 0.6))
    return FieldSpec(f"sel_{seed}", tuple(dims), "rel", eb,
                     {"kind": "grf", "beta": 3.0, "seed": seed, "zero_blocks": frac, "zero_edge": 16})


def workload_batch(count: int = 256, seed0: int = 100, scale: float = 1.0) -> list:
    """Uneven batch: ndim ~ U{1,2,3}; 1-D length log-uniform in [1e4, 3e8]; 2-D sides
    log-uniform up to 4096; 3-D up to 256x512x512; spectrum exponent U[2,4]; zero
    fraction U[0,0.5] in aligned blocks; eb from {1e-2,1e-3,1e-4}.  `scale` < 1
    shrinks every size (for tests)."""
    out = []
    for i in range(count):
        s = seed0 + i
        rng = np.random.default_rng(s)
        nd = int(rng.integers(1, 4))
        beta = float(rng.uniform(2.0, 4.0))
        zf = float(rng.uniform(0.0, 0.5))
        eb = float(rng.choice([1e-2, 1e-3, 1e-4]))

        def lu(lo, hi):
            return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        if nd == 1:
            dims = (max(16, int(lu(1e4, 3e8) * scale)),)
        elif nd == 2:
            dims = (max(8, int(lu(16, 4096) * math.sqrt(scale))), max(8, int(lu(16, 4096) * math.sqrt(scale))))
        else:
            c = scale ** (1.0 / 3.0)
            dims = (max(4, int(lu(8, 256) * c)), max(4, int(lu(8, 512) * c)), max(4, int(lu(8, 512) * c)))
        out.append(FieldSpec(f"batch_{s}", dims, "rel", eb,
                             {"kind": "grf", "beta": beta, "seed": s, "zero_blocks": zf,
                              "zero_edge": 16 if nd == 3 else 64}))
    return out
