"""Seeded synthetic inputs: sound-speed phantoms, transducer rings and grids.

This module only *creates inputs*. It holds none of the ray-tracing
arithmetic (no interpolation, no ray equations, no linking, no quadrature),
so both the CUDA path and the FP64 CPU oracle can be fed from it without
sharing any of the method's code.

Units: lengths in mm, sound speed in m/s (the library converts to mm/us).
Grid convention: node (i, j) sits at (x0 + i*h, y0 + j*h) with the grid
centred on the origin, x0 = -(nx-1)*h/2, y0 = -(ny-1)*h/2, and node (i, j) is
stored row-major at index j*nx + i.

Randomness comes from splitmix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), implemented here on numpy
uint64 arrays so that every machine draws the same numbers.

The paper's own workloads are measured breast data (URMC in-vitro/in-vivo)
and a k-Wave simulated set (Sec. 1, Sec. 5); none is available offline, so the
phantoms below stand in for them with breast-like sound speeds
(1400-1600 m/s) on a ring array, as the paper's ring geometry describes
(Sec. 1: one emitter fires at a time, all other elements receive).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based splitmix64 stream; ``uniform(n)`` gives doubles in [0, 1)."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, n: int) -> np.ndarray:
        k = np.arange(1, n + 1, dtype=np.uint64)
        with np.errstate(over="ignore"):
            z = self.state + k * _GOLDEN
            self.state = self.state + np.uint64(n) * _GOLDEN
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.next_u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int, sigma: float = 1.0) -> np.ndarray:
        """Box-Muller from two uniform draws per pair of outputs."""
        m = (n + 1) // 2
        u1 = self.uniform(m)
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log1p(-u1))
        z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
        return sigma * z[:n]

    def disc_points(self, n: int, radius: float) -> np.ndarray:
        """Uniform points in a disc (area-uniform radius)."""
        r = radius * np.sqrt(self.uniform(n))
        a = self.uniform(n, 0.0, 2 * np.pi)
        return np.stack([r * np.cos(a), r * np.sin(a)], axis=1)


@dataclasses.dataclass(frozen=True)
class Grid:
    nx: int
    ny: int
    h: float

    @property
    def x0(self) -> float:
        return -(self.nx - 1) * self.h / 2.0

    @property
    def y0(self) -> float:
        return -(self.ny - 1) * self.h / 2.0

    def node_xy(self):
        x = self.x0 + self.h * np.arange(self.nx)
        y = self.y0 + self.h * np.arange(self.ny)
        return np.meshgrid(x, y, indexing="xy")  # arrays [ny, nx]


def ring(n_tx: int, radius: float) -> np.ndarray:
    """Transducer k at angle 2*pi*k/N, counter-clockwise from +x; shape [N, 2]."""
    a = 2.0 * np.pi * np.arange(n_tx) / n_tx
    return np.stack([radius * np.cos(a), radius * np.sin(a)], axis=1)


def all_pairs(n_tx: int) -> np.ndarray:
    """All (e, r) with e != r, emitter-major; shape [N(N-1), 2] int32."""
    e = np.repeat(np.arange(n_tx), n_tx - 1)
    rr = np.tile(np.arange(n_tx - 1), n_tx)
    r = rr + (rr >= e)
    return np.stack([e, r], axis=1).astype(np.int32)


def homogeneous(grid: Grid, c: float = 1500.0) -> np.ndarray:
    return np.full((grid.ny, grid.nx), float(c))


def linear_gradient(grid: Grid, c_mid: float = 1500.0, g: float = 1.0) -> np.ndarray:
    """c = c_mid + g*y (g in (m/s)/mm)."""
    _, y = grid.node_xy()
    return c_mid + g * y


def fisheye(grid: Grid, c0: float = 1500.0, radius: float = 40.0) -> np.ndarray:
    """Maxwell fish-eye sound speed c0*(1 + r^2/R^2)/2, i.e. n = 2/(1 + r^2/R^2)."""
    x, y = grid.node_xy()
    return c0 * (1.0 + (x * x + y * y) / radius**2) / 2.0


def gaussian_inclusions(grid: Grid, seed: int, n_incl: int = 3, c_bg: float = 1500.0,
                        amp: float = 0.05, sigma_lo: float = 2.0, sigma_hi: float = 6.0,
                        centre_radius: float = 18.0) -> np.ndarray:
    """Background plus Gaussian blobs of relative amplitude +-amp (random sign)."""
    rng = SplitMix64(seed)
    sign = np.where(rng.uniform(n_incl) < 0.5, -1.0, 1.0)
    sig = rng.uniform(n_incl, sigma_lo, sigma_hi)
    mu = rng.disc_points(n_incl, centre_radius)
    x, y = grid.node_xy()
    rel = np.zeros_like(x)
    for k in range(n_incl):
        d2 = (x - mu[k, 0]) ** 2 + (y - mu[k, 1]) ** 2
        rel += sign[k] * amp * np.exp(-d2 / (2.0 * sig[k] ** 2))
    return c_bg * (1.0 + rel)


def gaussian_smooth(img: np.ndarray, sigma_px: float) -> np.ndarray:
    """Separable Gaussian blur (truncated at 4 sigma, edge-replicated), FP64."""
    r = int(math.ceil(4.0 * sigma_px))
    t = np.arange(-r, r + 1, dtype=np.float64)
    w = np.exp(-0.5 * (t / sigma_px) ** 2)
    w /= w.sum()
    out = img.astype(np.float64)
    for axis in (0, 1):
        pad = [(0, 0), (0, 0)]
        pad[axis] = (r, r)
        p = np.pad(out, pad, mode="edge")
        acc = np.zeros_like(out)
        n = out.shape[axis]
        for k in range(2 * r + 1):
            sl = [slice(None), slice(None)]
            sl[axis] = slice(k, k + n)
            acc += w[k] * p[tuple(sl)]
        out = acc
    return out


def breast_phantom(grid: Grid, seed: int, n_ell: int = 40, c_bg: float = 1480.0,
                   c_lo: float = 1400.0, c_hi: float = 1600.0, axis_lo: float = 2.0,
                   axis_hi: float = 15.0, centre_radius: float = 70.0,
                   smooth_mm: float = 1.0) -> np.ndarray:
    """Ellipses painted in seeded order on a background, then Gaussian-smoothed."""
    rng = SplitMix64(seed)
    cval = rng.uniform(n_ell, c_lo, c_hi)
    ax = rng.uniform(n_ell, axis_lo, axis_hi)
    ay = rng.uniform(n_ell, axis_lo, axis_hi)
    rot = rng.uniform(n_ell, 0.0, np.pi)
    mu = rng.disc_points(n_ell, centre_radius)
    x, y = grid.node_xy()
    img = np.full_like(x, c_bg)
    for k in range(n_ell):
        ca, sa = math.cos(rot[k]), math.sin(rot[k])
        u = (x - mu[k, 0]) * ca + (y - mu[k, 1]) * sa
        v = -(x - mu[k, 0]) * sa + (y - mu[k, 1]) * ca
        img[(u / ax[k]) ** 2 + (v / ay[k]) ** 2 <= 1.0] = cval[k]
    return gaussian_smooth(img, smooth_mm / grid.h)


@dataclasses.dataclass
class Workload:
    """One ToF problem: grid, sound speed(s), ring and stepping parameters."""
    name: str
    grid: Grid
    c: np.ndarray              # model sound speed [ny, nx] m/s
    tx: np.ndarray             # transducer positions [N, 2] mm
    ring_radius: float
    ds: float
    tol: float = 1e-4
    c_true: np.ndarray | None = None   # "measured" medium (inversion step)

    @property
    def n_tx(self) -> int:
        return int(self.tx.shape[0])

    @property
    def n_pairs(self) -> int:
        return self.n_tx * (self.n_tx - 1)


def cfg_small(seed: int = 1, n: int = 128, n_tx: int = 64) -> Workload:
    """128^2 grid at 0.5 mm, 3 Gaussian inclusions (+-5%, sigma 2-6 mm), 64-ring at 30 mm."""
    g = Grid(n, n, 0.5)
    R = 30.0
    c = gaussian_inclusions(g, seed, centre_radius=0.6 * R)
    return Workload("gauss3_128_ring64", g, c, ring(n_tx, R), R, ds=0.05)


def cfg_fisheye(n: int = 512, n_tx: int = 256, h: float = 0.2, ring_radius: float = 45.0,
                ds: float = 0.02) -> Workload:
    """Maxwell fish-eye c0(1+r^2/R^2)/2, c0=1500 m/s, R=40 mm; 512^2 at 0.2 mm; 256-ring at 45 mm."""
    g = Grid(n, n, h)
    return Workload("fisheye_512_ring256", g, fisheye(g), ring(n_tx, ring_radius), ring_radius, ds=ds)


def cfg_breast(seed: int = 3, n: int = 1024, n_tx: int = 512, h: float = 0.2,
               ring_radius: float = 95.0, ds: float = 0.02) -> Workload:
    """Breast-like 1024^2 at 0.2 mm: c_true = 40 smoothed ellipses (sigma 1 mm),
    c_model = c_true smoothed again with sigma 3 mm; 512-ring at 95 mm, step 0.02 mm."""
    g = Grid(n, n, h)
    scale = ring_radius / 95.0
    c_true = breast_phantom(g, seed, centre_radius=70.0 * scale,
                            axis_lo=2.0 * scale, axis_hi=15.0 * scale)
    c_model = gaussian_smooth(c_true, 3.0 / h)
    return Workload("breast_1024_ring512", g, c_model, ring(n_tx, ring_radius), ring_radius,
                    ds=ds, c_true=c_true)


def cfg_batch(seed: int = 4, n_inst: int = 32, sizes=(256, 512, 768, 1024),
              rings=(64, 128, 256, 512), h: float = 0.2, ds: float = 0.02) -> list[Workload]:
    """Uneven instances: grid side and ring size drawn uniformly; R_ring = 0.45*n*h;
    3 Gaussian inclusions scaled to the ring."""
    rng = SplitMix64(seed)
    pick_n = rng.uniform(n_inst)
    pick_r = rng.uniform(n_inst)
    out = []
    for k in range(n_inst):
        n = sizes[min(int(pick_n[k] * len(sizes)), len(sizes) - 1)]
        nt = rings[min(int(pick_r[k] * len(rings)), len(rings) - 1)]
        g = Grid(n, n, h)
        R = 0.45 * n * h
        sc = R / 30.0
        c = gaussian_inclusions(g, seed * 1000 + k, centre_radius=0.6 * R,
                                sigma_lo=2.0 * sc, sigma_hi=6.0 * sc)
        out.append(Workload(f"batch{k}_{n}_ring{nt}", g, c, ring(nt, R), R, ds=ds))
    return out


def born_perturbation(grid: Grid, ring_radius: float, seed: int = 5, sigma: float = 5.0) -> np.ndarray:
    """delta-c ~ N(0, sigma m/s) i.i.d. on nodes strictly inside the ring, 0 outside."""
    rng = SplitMix64(seed)
    x, y = grid.node_xy()
    dc = rng.normal(grid.nx * grid.ny, sigma).reshape(grid.ny, grid.nx)
    dc[x * x + y * y >= ring_radius**2] = 0.0
    return dc


def absorption_map(c_mps: np.ndarray, base: float = 2.0e-8, contrast: float = 20.0,
                   c_ref: float = 1500.0) -> np.ndarray:
    """A tissue-like absorption coefficient alpha0 (Np (rad/s)^-y m^-1) that
    follows the sound-speed structure: base * (1 + contrast |c/c_ref - 1|)
    (with y = 1.3, base 2e-8 is about 1 Np per 10 cm at 1 MHz; a 3 % inclusion
    absorbs 1.6x more)."""
    return base * (1.0 + contrast * np.abs(np.asarray(c_mps) / c_ref - 1.0))


@dataclasses.dataclass
class BornWorkload:
    """One ray-Born problem: background medium and ring (for the fan maps),
    the fan size, the frequencies and a sound-speed perturbation."""
    name: str
    grid: Grid
    c: np.ndarray              # background sound speed [ny, nx] m/s
    tx: np.ndarray             # transducer positions [N, 2] mm
    ring_radius: float
    ds: float
    fan_rays: int              # rays per transducer fan
    f_mhz: np.ndarray          # frequencies, MHz
    dc: np.ndarray             # perturbation [ny, nx] m/s, 0 outside the ring

    @property
    def n_tx(self) -> int:
        return int(self.tx.shape[0])


def born_fan_rays(ring_radius: float, h: float, multiple: int = 64) -> int:
    """Fan size K >= 2 pi * 2R / h (far-side ray spacing below one grid step),
    rounded up to a multiple of `multiple`."""
    k = math.ceil(2.0 * math.pi * 2.0 * ring_radius / h)
    return int(multiple * math.ceil(k / multiple))


def born_frequencies(n: int = 8, lo: float = 0.5, hi: float = 1.5) -> np.ndarray:
    return np.linspace(lo, hi, n)


def cfg_born(seed: int = 3, n: int = 1024, n_tx: int = 512, h: float = 0.2,
             ring_radius: float = 95.0, ds: float = 0.02) -> BornWorkload:
    """Ray-Born at full size: the breast model medium (1024^2 at 0.2 mm, 512-ring
    at 95 mm), 8 frequencies 0.5-1.5 MHz, dc ~ N(0, 5 m/s) inside the ring."""
    w = cfg_breast(seed, n, n_tx, h, ring_radius, ds)
    return BornWorkload("born_breast_1024_ring512", w.grid, w.c, w.tx, ring_radius, ds,
                        born_fan_rays(ring_radius, h), born_frequencies(),
                        born_perturbation(w.grid, ring_radius, seed=5))


def cfg_born_small(seed: int = 6, n: int = 128, n_tx: int = 64, h: float = 0.5,
                   ring_radius: float = 30.0, ds: float = 0.05) -> BornWorkload:
    """Scaled-down ray-Born: 128^2 at 0.5 mm, 64-ring at 30 mm, 3 broad Gaussian
    inclusions (+-3%, sigma 4-8 mm), 8 frequencies 0.5-1.5 MHz."""
    g = Grid(n, n, h)
    c = gaussian_inclusions(g, seed, amp=0.03, sigma_lo=4.0, sigma_hi=8.0,
                            centre_radius=0.6 * ring_radius)
    return BornWorkload("born_gauss3_128_ring64", g, c, ring(n_tx, ring_radius), ring_radius, ds,
                        born_fan_rays(ring_radius, h), born_frequencies(),
                        born_perturbation(g, ring_radius, seed=seed + 1))
