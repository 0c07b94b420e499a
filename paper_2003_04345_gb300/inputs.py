"""Seeded synthetic inputs: potentials, initial wavefunctions and workloads.

This module holds none of the integrator's arithmetic.  It only makes the
inputs that both the CUDA path and the CPU oracle consume (the potential V,
the initial state psi, chi per ensemble member), so that the two sides see
identical data.  It imports neither the CUDA binding nor the oracle.

Random numbers come from SplitMix64 (G. L. Steele, D. Lea, C. H. Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), used in its
counter form: output i of a stream with key k is mix64(k + (i+1) * gamma).

Workload shapes follow the paper's problem class (Sec. 2.1 and the
delta-potential experiment of Sec. 3.2): a periodic grid with nearest-neighbour
hopping, uniform on-site disorder plus a few strong defect sites, a cubic
nonlinearity, and a normalised Gaussian wavepacket with a plane-wave factor.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream identifiers, so that V, the defect positions and chi draw
# independent numbers from the same seed.
STREAM_DISORDER = 1
STREAM_DEFECTS = 2
STREAM_CHI = 3
STREAM_TRACE = 4


def mix64(z):
    """SplitMix64 finaliser on uint64 numpy values (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(state0, n):
    """The first n outputs of a SplitMix64 generator started at state0."""
    i = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        s = np.uint64(state0) + i * _GAMMA
    return mix64(s)


def stream_key(seed, stream):
    with np.errstate(over="ignore"):
        return mix64(np.uint64(seed) * _GAMMA + np.uint64(stream))[()]


def uniform(seed, stream, n):
    """n doubles in [0, 1) from stream ``stream`` of ``seed`` (53-bit mantissa)."""
    z = splitmix64(stream_key(seed, stream), n)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def defect_sites(S, n_defects, seed):
    """The first n_defects distinct site indices drawn from the defect stream."""
    if n_defects <= 0:
        return np.zeros(0, dtype=np.int64)
    if n_defects > S:
        raise ValueError("more defects than sites")
    chosen, seen = [], set()
    draw = 0
    batch = max(64, 2 * n_defects)
    while len(chosen) < n_defects:
        xs = uniform(seed, STREAM_DEFECTS, draw + batch)[draw:]
        draw += batch
        for x in xs:
            k = min(int(x * S), S - 1)
            if k not in seen:
                seen.add(k)
                chosen.append(k)
                if len(chosen) == n_defects:
                    break
    return np.array(chosen, dtype=np.int64)


def potential(nx, ny, W, n_defects, V_defect, seed):
    """V_k = W (xi_k - 1/2) + V_defect [k in D]: uniform disorder of width W
    plus n_defects strong sites, row-major (k = y*nx + x)."""
    S = nx * ny
    V = W * (uniform(seed, STREAM_DISORDER, S) - 0.5)
    D = defect_sites(S, n_defects, seed)
    V[D] += V_defect
    return V


def delta_potential(nx, ny, V0):
    """The paper's delta-like potential: V = V0 at the origin, 0 elsewhere (Sec. 3.2)."""
    V = np.zeros(nx * ny)
    V[0] = V0
    return V


def chi_for_seed(seed, lo=0.0, hi=2.0):
    return float(lo + (hi - lo) * uniform(seed, STREAM_CHI, 1)[0])


def wavepacket(nx, ny, sigma, kx, ky, cx=None, cy=None):
    """Normalised Gaussian wavepacket psi ~ exp(-(dx^2+dy^2)/(4 sigma^2)) exp(i(kx x + ky y)),
    dx, dy the minimum-image displacements from (cx, cy) (default: the grid centre),
    so sigma is the standard deviation of |psi|^2.  Returns complex128 (S,)."""
    cx = nx // 2 if cx is None else cx
    cy = ny // 2 if cy is None else cy
    x = np.arange(nx)
    y = np.arange(ny)
    dx = (x - cx + nx // 2) % nx - nx // 2
    dy = (y - cy + ny // 2) % ny - ny // 2
    g = np.exp(-(dy[:, None] ** 2 + dx[None, :] ** 2) / (4.0 * sigma * sigma))
    ph = np.exp(1j * (kx * x[None, :] + ky * y[:, None]))
    psi = (g * ph).reshape(nx * ny)
    return psi / math.sqrt(math.fsum((np.abs(psi) ** 2).tolist()))


def paper_initial_state(nx, ny):
    """u(x, y) = 1 + 2 cos x + 2 cos y on [0, 2 pi)^2 (Sec. 3, parameter list)."""
    x = 2 * math.pi * np.arange(nx) / nx
    y = 2 * math.pi * np.arange(ny) / ny
    return (1 + 2 * np.cos(x)[None, :] + 2 * np.cos(y)[:, None]).reshape(nx * ny).astype(np.complex128)


def paper_laplacian_hopping(nx, ny, lx=2 * math.pi, ly=2 * math.pi):
    """(tx, ty, eps0) that make K the paper's 5-point -Laplacian (eq. Kdefinition)."""
    hx, hy = lx / nx, ly / ny
    tx, ty = 1.0 / hx ** 2, 1.0 / hy ** 2
    return tx, ty, 2 * tx + 2 * ty


@dataclass
class Workload:
    """One synthetic instance: grid, physics, initial state recipe, step count."""
    name: str
    nx: int
    ny: int
    h: float
    steps: int
    chi: float = 1.0
    W: float = 1.0
    defect_fraction: float = 0.0
    n_defects: int | None = None
    V_defect: float = 20.0
    sigma: float = 2.0
    kx: float = math.pi / 4
    ky: float = 0.0
    tx: float = 1.0
    ty: float = 1.0
    eps0: float = 0.0
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def S(self):
        return self.nx * self.ny

    def defects(self):
        if self.n_defects is not None:
            return self.n_defects
        return int(round(self.defect_fraction * self.S))

    def potential(self):
        return potential(self.nx, self.ny, self.W, self.defects(), self.V_defect, self.seed)

    def psi0(self):
        return wavepacket(self.nx, self.ny, self.sigma, self.kx, self.ky)

    def as_dict(self):
        d = asdict(self)
        d["defects"] = self.defects()
        return d


def grid16_fp64():
    """16x16, W=1, 3 defects at V=20, chi=1, sigma=2, k=(pi/4,0), h=0.01, 100 steps."""
    return Workload("grid16_fp64", 16, 16, h=0.01, steps=100, chi=1.0, W=1.0, n_defects=3,
                    sigma=2.0)


def grid512_fp64():
    """512x512, W=1, 1% defects at V=20, chi=1, sigma=8, h=0.005, 1000 steps."""
    return Workload("grid512_fp64", 512, 512, h=0.005, steps=1000, chi=1.0, W=1.0,
                    defect_fraction=0.01, sigma=8.0)


def grid2048_mixed():
    """2048x2048, W=2, 1% defects, chi=2, sigma=8, h=0.002, 500 steps."""
    return Workload("grid2048_mixed", 2048, 2048, h=0.002, steps=500, chi=2.0, W=2.0,
                    defect_fraction=0.01, sigma=8.0)


def grid128_crop_of_2048():
    """128x128 instance with the 2048x2048 physics (the size the oracle can follow)."""
    return Workload("grid128_2048physics", 128, 128, h=0.002, steps=500, chi=2.0, W=2.0,
                    defect_fraction=0.01, sigma=8.0)


def ensemble128(seed):
    """One member of the 1024-member 128x128 ensemble: chi ~ U[0,2] from the seed."""
    return Workload(f"ensemble128_seed{seed}", 128, 128, h=0.01, steps=2000,
                    chi=chi_for_seed(seed), W=1.0, defect_fraction=0.01, sigma=8.0, seed=seed)


def served_trace(n_requests, rate_hz, seed=0, sizes=(64, 128, 256, 512, 1024),
                 steps_range=(100, 5000), hs=(0.002, 0.005, 0.01), max_defect_fraction=0.02):
    """Poisson arrivals (exponential gaps of mean 1/rate_hz) of simulation requests
    with grid size, step count, h, defect density and seed drawn per request."""
    u = uniform(seed, STREAM_TRACE, 6 * n_requests).reshape(n_requests, 6)
    t = 0.0
    reqs = []
    for r in range(n_requests):
        t += -math.log(1.0 - u[r, 0]) / rate_hz
        n = sizes[min(int(u[r, 1] * len(sizes)), len(sizes) - 1)]
        lo, hi = steps_range
        steps = lo + min(int(u[r, 2] * (hi - lo + 1)), hi - lo)
        h = hs[min(int(u[r, 3] * len(hs)), len(hs) - 1)]
        frac = max_defect_fraction * u[r, 4]
        rseed = int(u[r, 5] * 2 ** 31)
        w = Workload(f"req{r}", n, n, h=h, steps=steps, chi=1.0, W=1.0, defect_fraction=frac,
                     sigma=8.0, seed=rseed)
        reqs.append((t, w))
    return reqs
