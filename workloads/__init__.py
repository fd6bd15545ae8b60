"""Seeded synthetic inputs for the acoustic wave-step workloads.

This module only *makes inputs*: padded fields, velocity models, source
wavelets, source/receiver positions and the time step from a CFL number.  It
holds none of the method's arithmetic (no stencil, no leapfrog update, no
source scaling), so that both the CUDA path and the FP64 oracle can be fed the
same numbers without sharing any code that computes a result.

Layout convention (the paper flattens each grid to 1D with halo padding,
Sec. 11.3 "GPU Code Generation"): a padded field of interior ``nx*ny*nz`` and
halo width ``halo`` is a C-contiguous array of shape
``(nz + 2*halo, ny + 2*halo, nx + 2*halo)`` -- x fastest, z slowest (the
streamed axis).  Interior point ``(i, j, k)`` sits at padded index
``(k + halo, j + halo, i + halo)``; its *interior linear index* is
``i + nx*(j + ny*k)``.

Random numbers come from ``numpy.random.default_rng(seed)`` (PCG64), which is
bit-identical on x86-64 and aarch64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Seed base for the synthetic workloads (arXiv 2309.04671 -> 23090467).
SEED_BASE = 23090467


def padded_shape(nx: int, ny: int, nz: int, halo: int) -> tuple[int, int, int]:
    return (nz + 2 * halo, ny + 2 * halo, nx + 2 * halo)


def interior(a: np.ndarray, halo: int) -> np.ndarray:
    """View of the interior of a padded field."""
    h = halo
    return a[h:a.shape[0] - h, h:a.shape[1] - h, h:a.shape[2] - h]


def linear_index(i, j, k, nx: int, ny: int):
    """Interior linear index of interior point (i, j, k)."""
    return np.asarray(i, np.int64) + nx * (np.asarray(j, np.int64) + ny * np.asarray(k, np.int64))


def uniform_field(nx, ny, nz, halo, seed, *, halo_random=True, dtype=np.float32):
    """Uniform[-1, 1] field on the padded grid.

    With ``halo_random`` the halo holds random values too (a stencil reads the
    halo "as given"); otherwise the halo is zero (Dirichlet wave fields).
    """
    rng = np.random.default_rng(seed)
    shape = padded_shape(nx, ny, nz, halo)
    a = np.empty(shape, dtype=dtype)
    # fill slab by slab to bound the float64 temporary at large sizes
    for z0 in range(0, shape[0], 16):
        z1 = min(shape[0], z0 + 16)
        a[z0:z1] = rng.uniform(-1.0, 1.0, size=(z1 - z0,) + shape[1:])
    if not halo_random and halo > 0:
        zero_halo(a, halo)
    return a


def zero_halo(a: np.ndarray, halo: int) -> np.ndarray:
    h = halo
    if h == 0:
        return a
    a[:h] = 0
    a[-h:] = 0
    a[:, :h] = 0
    a[:, -h:] = 0
    a[:, :, :h] = 0
    a[:, :, -h:] = 0
    return a


@dataclass
class Gaussians:
    centre: np.ndarray   # (G, 3) interior coordinates (x, y, z), in cells
    amp: np.ndarray      # (G,)
    sigma: np.ndarray    # (G,) in cells


def layered_velocity(nx, ny, nz, halo, seed, *, nlayers=8, vmin=1500.0, vmax=4500.0,
                     ngauss=16, amp=0.10, dtype=np.float32, return_params=False):
    """Layered velocity model with Gaussian perturbations.

    ``nlayers`` equal-thickness z-layers with v_k = vmin + k*(vmax-vmin)/(nlayers-1),
    multiplied by (1 + sum_i a_i exp(-|x-c_i|^2 / (2 sigma_i^2))) with
    centres uniform over the interior, a_i ~ U[-amp, amp] and
    sigma_i ~ U[n/32, n/8] cells (n = min(nx, ny, nz)).  The halo repeats the
    nearest interior value (a wave step never reads velocity in the halo).
    """
    rng = np.random.default_rng(seed)
    n = min(nx, ny, nz)
    g = Gaussians(
        centre=np.stack([rng.uniform(0, nx - 1, ngauss), rng.uniform(0, ny - 1, ngauss),
                         rng.uniform(0, nz - 1, ngauss)], axis=1),
        amp=rng.uniform(-amp, amp, ngauss),
        sigma=rng.uniform(n / 32.0, n / 8.0, ngauss),
    )
    xs = np.arange(nx, dtype=np.float64)
    ys = np.arange(ny, dtype=np.float64)
    zs = np.arange(nz, dtype=np.float64)
    gx = [np.exp(-(xs - g.centre[q, 0]) ** 2 / (2 * g.sigma[q] ** 2)) for q in range(ngauss)]
    gy = [np.exp(-(ys - g.centre[q, 1]) ** 2 / (2 * g.sigma[q] ** 2)) for q in range(ngauss)]
    gz = [np.exp(-(zs - g.centre[q, 2]) ** 2 / (2 * g.sigma[q] ** 2)) for q in range(ngauss)]
    layer = np.minimum((np.arange(nz) * nlayers) // nz, nlayers - 1)
    vlayer = vmin + layer * (vmax - vmin) / (nlayers - 1)

    shape = padded_shape(nx, ny, nz, halo)
    v = np.empty(shape, dtype=dtype)
    h = halo
    slab = max(1, (1 << 24) // max(1, nx * ny))
    for z0 in range(0, nz, slab):
        z1 = min(nz, z0 + slab)
        pert = np.ones((z1 - z0, ny, nx), dtype=np.float64)
        for q in range(ngauss):
            pert += g.amp[q] * (gz[q][z0:z1, None, None] * (gy[q][None, :, None] * gx[q][None, None, :]))
        pert *= vlayer[z0:z1, None, None]
        v[z0 + h:z1 + h, h:ny + h, h:nx + h] = pert
    _edge_fill_halo(v, h)
    if return_params:
        return v, g
    return v


def layered_velocity_torch(nx, ny, nz, halo, seed, device, *, nlayers=8, vmin=1500.0, vmax=4500.0, ngauss=16,
                           amp=0.10):
    """The same recipe as :func:`layered_velocity` (same random parameters
    for the same seed), evaluated with torch on ``device`` in FP64 and
    returned as an FP32 tensor; for inputs too large to generate quickly on
    the host.  Values can differ from the NumPy version in the last bits."""
    import torch
    rng = np.random.default_rng(seed)
    n = min(nx, ny, nz)
    centre = np.stack([rng.uniform(0, nx - 1, ngauss), rng.uniform(0, ny - 1, ngauss),
                       rng.uniform(0, nz - 1, ngauss)], axis=1)
    a = rng.uniform(-amp, amp, ngauss)
    sigma = rng.uniform(n / 32.0, n / 8.0, ngauss)
    f64 = dict(dtype=torch.float64, device=device)
    xs, ys, zs = (torch.arange(m, **f64) for m in (nx, ny, nz))
    layer = torch.clamp((torch.arange(nz, device=device) * nlayers) // nz, max=nlayers - 1).to(torch.float64)
    vlayer = vmin + layer * (vmax - vmin) / (nlayers - 1)
    pert = torch.ones((nz, ny, nx), **f64)
    for q in range(ngauss):
        gx = torch.exp(-(xs - centre[q, 0]) ** 2 / (2 * sigma[q] ** 2))
        gy = torch.exp(-(ys - centre[q, 1]) ** 2 / (2 * sigma[q] ** 2))
        gz = torch.exp(-(zs - centre[q, 2]) ** 2 / (2 * sigma[q] ** 2))
        pert += a[q] * (gz[:, None, None] * (gy[None, :, None] * gx[None, None, :]))
    pert *= vlayer[:, None, None]
    v = torch.nn.functional.pad(pert.to(torch.float32)[None, None], (halo,) * 6, mode="replicate")[0, 0]
    return v.contiguous()


@dataclass
class ShotSpec:
    """One shot of a batch: interior sizes, velocity seed, source cell, h, CFL."""
    nx: int
    ny: int
    nz: int
    vel_seed: int
    src: tuple
    h: float = 10.0
    cfl: float = 0.4


def batch_specs(nshots: int = 64, lo: int = 96, hi: int = 320, seed_offset: int = 4,
                src_depth: int = 8) -> list:
    """Shots with side lengths uniform in [lo, hi] per axis (seeded), each
    with its own layered velocity seed and a source at a seeded surface
    position ``src_depth`` cells deep."""
    rng = np.random.default_rng(SEED_BASE + seed_offset)
    out = []
    for s in range(nshots):
        nx, ny, nz = (int(v) for v in rng.integers(lo, hi + 1, 3))
        i, j = int(rng.integers(0, nx)), int(rng.integers(0, ny))
        out.append(ShotSpec(nx, ny, nz, SEED_BASE + 1000 + s + 1000 * seed_offset, (i, j, min(src_depth, nz - 1))))
    return out


def _edge_fill_halo(a: np.ndarray, h: int) -> None:
    if h == 0:
        return
    a[:h] = a[h:h + 1]
    a[-h:] = a[-h - 1:-h]
    a[:, :h] = a[:, h:h + 1]
    a[:, -h:] = a[:, -h - 1:-h]
    a[:, :, :h] = a[:, :, h:h + 1]
    a[:, :, -h:] = a[:, :, -h - 1:-h]


def constant_velocity(nx, ny, nz, halo, v=1500.0, dtype=np.float32):
    return np.full(padded_shape(nx, ny, nz, halo), v, dtype=dtype)


def ricker(nt: int, dt: float, f: float = 15.0, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet r(t_n), t_n = n*dt, peak amplitude 1 at t0 (default 1/f).

    r(t) = (1 - 2 pi^2 f^2 (t - t0)^2) exp(-pi^2 f^2 (t - t0)^2), computed in
    float64 on the host.  It is the source's time function, an input: the
    paper leaves the source signature to the user.
    """
    if t0 is None:
        t0 = 1.0 / f
    t = np.arange(nt, dtype=np.float64) * dt - t0
    a = (math.pi * f * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def dt_for_cfl(cfl: float, h: float, vmax: float) -> float:
    """Time step giving CFL = vmax*dt/h."""
    return cfl * h / vmax


@dataclass
class WaveProblem:
    """One acoustic wave-propagation workload (interior sizes, halo, inputs)."""
    name: str
    nx: int
    ny: int
    nz: int
    halo: int
    h: float
    dt: float
    nsteps: int
    vel: np.ndarray                  # float32 padded
    src_idx: np.ndarray              # int64 interior linear indices (nsrc,)
    src_amp: np.ndarray              # float32 (nt, nsrc): f^n, unscaled source function
    rec_idx: np.ndarray = field(default_factory=lambda: np.zeros(0, np.int64))
    meta: dict = field(default_factory=dict)

    @property
    def npoints(self) -> int:
        return self.nx * self.ny * self.nz


def small_constant_problem(n: int = 64, nsteps: int = 20, halo: int = 4) -> WaveProblem:
    """64^3 interior, h=10 m, v=1500 m/s, dt=1 ms, 15 Hz Ricker at the grid centre."""
    h, dt = 10.0, 1e-3
    vel = constant_velocity(n, n, n, halo, 1500.0)
    src = linear_index(n // 2, n // 2, n // 2, n, n).reshape(1)
    amp = ricker(nsteps, dt, 15.0).astype(np.float32).reshape(nsteps, 1)
    return WaveProblem(f"const{n}", n, n, n, halo, h, dt, nsteps, vel, src, amp,
                       meta={"v": 1500.0, "cfl": 1500.0 * dt / h})


def layered_problem(n: int = 512, nsteps: int = 100, halo: int = 4, cfl: float = 0.4,
                    seed_offset: int = 2, src_depth: int = 20, ny: int | None = None,
                    nz: int | None = None) -> WaveProblem:
    """Layered + 16-Gaussian velocity, h=10 m, dt at CFL 0.4, 15 Hz Ricker at depth 20."""
    nx = n
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    h = 10.0
    vel = layered_velocity(nx, ny, nz, halo, SEED_BASE + seed_offset)
    vmax = float(interior(vel, halo).max())
    dt = dt_for_cfl(cfl, h, vmax)
    src = linear_index(nx // 2, ny // 2, min(src_depth, nz - 1), nx, ny).reshape(1)
    amp = ricker(nsteps, dt, 15.0).astype(np.float32).reshape(nsteps, 1)
    return WaveProblem(f"layered{nx}x{ny}x{nz}", nx, ny, nz, halo, h, dt, nsteps, vel, src, amp,
                       meta={"vmax": vmax, "cfl": cfl})
