"""Seeded synthetic inputs for the acoustic wave path.

This module holds no arithmetic of the method itself (no stencil, no FD
weights, no damping, no interpolation): it only draws the inputs that both the
CUDA path and the FP64 oracle consume, so the same arrays feed both sides.

The paper's workloads are Devito's acoustic example (McCormick 2017, Section
"Acoustic wave equation": SO8, FP32, grids 256^3-512^3) and a Gaussian initial
field (Section "Functional Correctness", Fig. guassian_init).  There is no
dataset; everything here is synthetic and seeded.

Random numbers: SplitMix64 (Steele, Lea, Flood 2014) for uniform doubles in
[0, 1) from the top 53 bits, Box-Muller for normals.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int) -> np.ndarray:
    """n consecutive SplitMix64 outputs of a generator started at ``seed``."""
    with np.errstate(over="ignore"):
        state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + _GOLDEN * np.arange(1, n + 1, dtype=np.uint64)
        z = state
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normals by Box-Muller on pairs of SplitMix64 uniforms."""
    k = (n + 1) // 2
    u = uniform(seed, 2 * k)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * k)
    out[0::2] = rad * np.cos(2.0 * math.pi * u2)
    out[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return out[:n]


def gaussian_blur(a: np.ndarray, sigma: float) -> np.ndarray:
    """Separable Gaussian blur, truncated at 3 sigma, zero padding."""
    from scipy.ndimage import gaussian_filter1d

    out = np.asarray(a, dtype=np.float32)
    for ax in range(out.ndim):
        out = gaussian_filter1d(out, sigma, axis=ax, mode="constant", cval=0.0, truncate=3.0)
    return out


def layered_velocity(shape, nlayers=20, vmin=1.5, vmax=4.5) -> np.ndarray:
    """Velocity (km/s) of ``nlayers`` equal-thickness layers stacked along z
    (the depth axis), v_k = vmin + (vmax - vmin) k / (nlayers - 1)."""
    nx, ny, nz = shape
    k = np.minimum((np.arange(nz) * nlayers) // nz, nlayers - 1)
    vz = vmin + (vmax - vmin) * k / max(nlayers - 1, 1)
    return np.broadcast_to(vz.astype(np.float32), (nx, ny, nz))


def velocity_model(shape, seed: int, *, nlayers=20, vmin=1.5, vmax=4.5, amp=0.05, sigma=5.0) -> np.ndarray:
    """20-layer model with a seeded +-5 % perturbation: iid N(0,1) blurred with
    sigma cells, normalised to max |p| = 1, v <- v (1 + amp p)."""
    n = int(np.prod(shape))
    p = normal(seed, n).astype(np.float32).reshape(shape)
    p = gaussian_blur(p, sigma)
    p /= np.max(np.abs(p))
    v = layered_velocity(shape, nlayers, vmin, vmax) * (1.0 + amp * p)
    return v.astype(np.float32)


def slowness2(v: np.ndarray) -> np.ndarray:
    """m = 1 / v^2 in (ms/m)^2 (v in km/s = m/ms), float32."""
    v = np.asarray(v, dtype=np.float64)
    return (1.0 / (v * v)).astype(np.float32)


def ricker(nt: int, dt: float, f: float, t0: float | None = None) -> np.ndarray:
    """Ricker wavelet sampled at t = n dt (ms), peak frequency f (Hz), delay
    t0 = 1/f, unit amplitude.  Row n feeds update n."""
    fk = f * 1e-3  # cycles per ms
    if t0 is None:
        t0 = 1.0 / fk
    t = np.arange(nt) * dt - t0
    a = (math.pi * fk * t) ** 2
    return ((1.0 - 2.0 * a) * np.exp(-a)).astype(np.float64)


# Spectral radius |a_0| + 2 sum |a_k| of the centred second-derivative stencil
# of order SO on unit spacing, as exact rationals.  Used only to choose a dt
# below the leapfrog stability limit for the synthetic workloads.
_RHO = {
    2: 4.0,
    4: 16.0 / 3.0,
    6: 272.0 / 45.0,
    8: 2048.0 / 315.0,
    10: 512.0 / 75.0,
    12: 367616.0 / 51975.0,
    14: 34374656.0 / 4729725.0,
    16: 35127296.0 / 4729725.0,
}


def _rho(so: int) -> float:
    return _RHO[so]


def cfl_dt(so: int, spacing, vmax: float, frac: float = 0.9) -> float:
    """frac x the leapfrog stability limit 2 / (vmax sqrt(sum_a rho / h_a^2)) (ms)."""
    s = sum(_rho(so) / (h * h) for h in spacing)
    return frac * 2.0 / (vmax * math.sqrt(s))


def gaussian_field(shape, sigma=0.4) -> np.ndarray:
    """Fig. guassian_init: a 3D normal pdf with standard deviation sigma on
    [-1, 1]^3, sampled at shape points (the paper's source-free initial u)."""
    axes = [np.linspace(-1.0, 1.0, n) for n in shape]
    x, y, z = np.meshgrid(*axes, indexing="ij")
    norm = 1.0 / ((2.0 * math.pi) ** 1.5 * sigma ** 3)
    return (norm * np.exp(-(x * x + y * y + z * z) / (2.0 * sigma * sigma))).astype(np.float32)


def surface_receivers(shape, spacing, n_side: int, depth: float) -> np.ndarray:
    """n_side x n_side receivers evenly spread over [0, (nx-1)hx] x [0, (ny-1)hy] at depth (m)."""
    xs = np.linspace(0.0, (shape[0] - 1) * spacing[0], n_side)
    ys = np.linspace(0.0, (shape[1] - 1) * spacing[1], n_side)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), np.full(X.size, float(depth))], axis=1)


def line_receivers(shape, spacing, n: int, depth: float, y_index=None) -> np.ndarray:
    """n receivers evenly spread along x at the centre y and the given depth (m)."""
    xs = np.linspace(0.0, (shape[0] - 1) * spacing[0], n)
    yc = (shape[1] // 2 if y_index is None else y_index) * spacing[1]
    return np.stack([xs, np.full(n, yc), np.full(n, float(depth))], axis=1)


@dataclass
class Workload:
    """One synthetic problem: grid, spacing, SO, dt, nt, model, source, receivers."""

    name: str
    shape: tuple
    spacing: tuple
    so: int
    nt: int
    dt: float
    m: np.ndarray
    src_xyz: np.ndarray
    wavelet: np.ndarray
    rec_xyz: np.ndarray
    sponge_width: int = 0
    sponge_faces: int = 0b101111
    vmax: float = 1.5
    extra: dict = field(default_factory=dict)

    @property
    def points(self) -> int:
        return int(np.prod(self.shape))


def plain_forward_64(nt: int = 50) -> Workload:
    """64^3, h = 10 m, SO4, v = 1.5 km/s, dt = 0.9 CFL, 10 Hz Ricker at the
    grid centre, zero Dirichlet, fields start at 0; one receiver at the source."""
    shape, h, so, v = (64, 64, 64), (10.0, 10.0, 10.0), 4, 1.5
    dt = cfl_dt(so, h, v)
    m = np.full(shape, 1.0 / (v * v), dtype=np.float32)
    src = np.array([[32 * h[0], 32 * h[1], 32 * h[2]]])
    wav = ricker(nt, dt, 10.0)[:, None]
    return Workload("plain_forward_64^3_so4", shape, h, so, nt, dt, m, src, wav, src.copy(), 0, 0b101111, v)


def layered_forward(shape=(512, 512, 512), so=8, nt=1000, seed=1, f=15.0, h=10.0,
                    sponge_width=10, nrec_line=0) -> Workload:
    """Layered 1.5-4.5 km/s model with a seeded +-5 % blurred perturbation,
    Ricker source at depth 20 m above the grid centre, 10-cell sponge on all
    faces but the top (z = 0)."""
    spacing = (h, h, h)
    v = velocity_model(shape, seed)
    vmax = 4.5 * 1.05
    dt = cfl_dt(so, spacing, vmax)
    src = np.array([[(shape[0] // 2) * h, (shape[1] // 2) * h, 20.0]])
    wav = ricker(nt, dt, f)[:, None]
    rec = line_receivers(shape, spacing, nrec_line, 20.0) if nrec_line else np.zeros((0, 3))
    return Workload("layered_%dx%dx%d_so%d" % (shape + (so,)), tuple(shape), spacing, so, nt, dt,
                    slowness2(v), src, wav, rec, sponge_width, 0b101111, vmax)


def tiled_forward_512(nt: int = 1000) -> Workload:
    """512^3, h = 10 m, SO8, 1000 steps, layered + perturbed model (seed 1),
    15 Hz Ricker at depth 20 m, 10-cell sponge."""
    return layered_forward((512, 512, 512), 8, nt, seed=1, f=15.0, h=10.0, sponge_width=10)


def high_order_forward(nt: int = 500, shape=(768, 768, 384), n_side=501) -> Workload:
    """768 x 768 x 384, h = 12.5 m, SO16, 500 steps, same recipe (seed 2),
    501 x 501 surface receivers at 25 m depth, trilinear."""
    w = layered_forward(shape, 16, nt, seed=2, f=15.0, h=12.5, sponge_width=10)
    w.rec_xyz = surface_receivers(shape, w.spacing, n_side, 25.0)
    w.name = "high_order_%dx%dx%d_so16" % tuple(shape)
    return w
