"""Seeded synthetic input fields shaped like the paper's workloads.

This module only draws inputs; it holds none of the reduction method's
arithmetic, so both the GPU path and the CPU oracle may use it.

The paper evaluates on NYX (512^3 FP32 cosmology), XGC and E3SM fields
(Sec. VI, Table III), which are not available here; these generators stand in
for them:

* ``sinusoid_field_2d`` -- sum of four sinusoids with random integer
  wavevectors |k| <= 8, amplitudes U(0.5, 1), phases U(0, 2 pi), plus
  N(0, 0.01^2) noise, on [0,1]^2 (the small case the oracle runs in seconds);
* ``powerlaw_field`` -- Gaussian random field with power spectrum
  P(k) ~ |k|^-11/3 (Kolmogorov-like, NYX-like roughness): complex white noise
  times sqrt(P), k = 0 removed, inverse real FFT, normalised to zero mean and
  unit variance;
* ``front_field`` -- a power-law field plus a tanh front of width 5 cells
  across the first axis (the host-resident streaming case);
* ``batch_shapes`` -- shapes and bounds of a batch of uneven fields.

numpy generators are the reference; ``powerlaw_field_torch`` draws the same
recipe on a CUDA device (different random numbers, same distribution) for
sizes where the host FFT would be slow.
"""
import math

import numpy as np

__all__ = ["sinusoid_field_2d", "powerlaw_field", "front_field", "batch_shapes",
           "powerlaw_field_torch", "front_field_torch", "random_coefficients"]


def sinusoid_field_2d(n=129, seed=0, dtype=np.float32):
    rng = np.random.default_rng(seed)
    x = np.linspace(0.0, 1.0, n)
    X, Y = np.meshgrid(x, x, indexing="ij")
    f = np.zeros((n, n))
    for _ in range(4):
        while True:
            k = rng.integers(-8, 9, size=2)
            if 0 < math.hypot(*k) <= 8:
                break
        a = rng.uniform(0.5, 1.0)
        phi = rng.uniform(0.0, 2 * math.pi)
        f += a * np.sin(2 * math.pi * (k[0] * X + k[1] * Y) + phi)
    f += rng.normal(0.0, 0.01, size=f.shape)
    return f.astype(dtype)


def _kgrid(shape):
    ks = [np.fft.fftfreq(n) * n for n in shape[:-1]] + [np.fft.rfftfreq(shape[-1]) * shape[-1]]
    k2 = np.zeros([len(k) for k in ks])
    for ax, k in enumerate(ks):
        sh = [1] * len(shape)
        sh[ax] = len(k)
        k2 = k2 + (k.reshape(sh) ** 2)
    return k2


def powerlaw_field(shape, seed=1, exponent=-11.0 / 3.0, dtype=np.float32):
    shape = tuple(int(s) for s in shape)
    rng = np.random.default_rng(seed)
    k2 = _kgrid(shape)
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (exponent / 4.0)          # sqrt(P(k)) = |k|^(exponent/2)
    noise = rng.standard_normal(k2.shape) + 1j * rng.standard_normal(k2.shape)
    f = np.fft.irfftn(noise * amp, s=shape, axes=tuple(range(len(shape))))
    f -= f.mean()
    f /= f.std()
    return f.astype(dtype)


def front_field(shape, seed=7, dtype=np.float32):
    f = powerlaw_field(shape, seed=seed, dtype=np.float64)
    x = np.arange(shape[0], dtype=np.float64) - (shape[0] - 1) / 2.0
    sh = [shape[0]] + [1] * (len(shape) - 1)
    f = f + np.tanh(x / 5.0).reshape(sh)
    return f.astype(dtype)


def batch_shapes(count=256, seed=3, lo=17, hi=513):
    """Shapes (2-D or 3-D with p = 1/2, dims log-uniform in [lo, hi]) and
    relative bounds drawn from {1e-2, 1e-3, 1e-4}."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        d = 2 if rng.random() < 0.5 else 3
        dims = tuple(int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
                     for _ in range(d))
        tol = float(rng.choice([1e-2, 1e-3, 1e-4]))
        out.append((dims, tol))
    return out


def random_coefficients(n, seed, scale=1.0):
    """Standard-normal values (e.g. a seeded stand-in coefficient stream)."""
    return np.random.default_rng(seed).standard_normal(n) * scale


def powerlaw_field_torch(shape, seed=1, exponent=-11.0 / 3.0, device="cuda", dtype=None):
    import torch
    shape = tuple(int(s) for s in shape)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    ks = [torch.fft.fftfreq(n, device=device, dtype=torch.float64) * n for n in shape[:-1]]
    ks.append(torch.fft.rfftfreq(shape[-1], device=device, dtype=torch.float64) * shape[-1])
    hs = [len(k) for k in ks]
    k2 = torch.zeros(hs, device=device, dtype=torch.float32)
    for ax, k in enumerate(ks):
        sh = [1] * len(shape)
        sh[ax] = len(k)
        k2 = k2 + (k.float().reshape(sh) ** 2)
    amp = torch.where(k2 > 0, k2.clamp_min(1e-30) ** (exponent / 4.0), torch.zeros_like(k2))
    del k2
    re = torch.randn(hs, generator=g, device=device, dtype=torch.float32)
    im = torch.randn(hs, generator=g, device=device, dtype=torch.float32)
    spec = torch.complex(re * amp, im * amp)
    del re, im, amp
    f = torch.fft.irfftn(spec, s=shape)
    del spec
    f = f - f.mean()
    f = f / f.std()
    return f.to(dtype or torch.float32).contiguous()


def front_field_torch(shape, seed=7, device="cuda"):
    import torch
    f = powerlaw_field_torch(shape, seed=seed, device=device)
    x = torch.arange(shape[0], device=device, dtype=torch.float32) - (shape[0] - 1) / 2.0
    f += torch.tanh(x / 5.0).reshape([shape[0]] + [1] * (len(shape) - 1))
    return f


def node_coords(shape, seed, kind="random"):
    """Strictly increasing node coordinates for every dimension of a
    non-uniform grid: "random" spacings drawn uniformly from [0.3, 2.5]
    (ratio up to about 8 between neighbouring cells), or "stretched" nodes
    clustered towards both ends as in a boundary-layer mesh
    (x = sinh(4 (t - 1/2)) on t uniform in [0, 1])."""
    rng = np.random.default_rng(seed)
    out = []
    for n in shape:
        if kind == "stretched":
            out.append(np.sinh(4.0 * (np.linspace(0.0, 1.0, n) - 0.5)))
        else:
            out.append(np.cumsum(rng.uniform(0.3, 2.5, size=n)))
    return out
