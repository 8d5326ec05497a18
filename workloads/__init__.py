"""Seeded synthetic particle sets shaped like the paper's in situ workloads.

This module only draws random numbers: it holds none of the binning
arithmetic. Both the CPU oracle and the CUDA path are fed from here, so the
two sides see the same bytes for the same seed.

The paper's own data (Newton++ uniform-random initial conditions with 24 M
bodies, MAGI galaxy models; Sec. 4.1 and 4.3) is not available, so these
generators stand in for it:

* ``uniform``    -- x, y ~ U[0,1)^2, mass ~ U[1,2], speed ~ |N(0,1)|
                    (the uniform random initial condition of Sec. 4.3).
* ``plummer``    -- a Plummer sphere of scale radius 1 truncated at r = 10,
                    projected onto x-y (a centrally concentrated body set,
                    standing in for the MAGI galaxy models of Sec. 4.1).
* ``gaussians``  -- a mixture of 16 isotropic Gaussians in [0,1)^2 with
                    log-uniform widths (clustered data that stresses
                    per-bin precision).
* ``batch``      -- many uneven simulation blocks, each with its own grid
                    (the many binning operations per step of Sec. 4.3).
* ``serving``    -- a Poisson stream of binning requests over a particle
                    pool (the asynchronous in situ method of Sec. 3).

Every generator uses numpy's PCG64 with an explicit seed.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

__all__ = [
    "Workload",
    "BatchPlan",
    "ServingPlan",
    "uniform",
    "plummer",
    "gaussians",
    "batch",
    "serving",
    "named",
]


@dataclasses.dataclass
class Workload:
    """One binning problem: SoA columns plus the grid they are binned onto."""

    name: str
    x: np.ndarray
    y: np.ndarray
    attrs: List[np.ndarray]
    lo: tuple
    hi: tuple
    res: tuple

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def dtype(self) -> np.dtype:
        return self.x.dtype

    def bytes_read(self) -> int:
        """Bytes of the coordinate and attribute columns (read once)."""
        return (2 + len(self.attrs)) * self.n * self.x.dtype.itemsize

    def bytes_written(self) -> int:
        """Bytes of the per-bin outputs: count u64, then per attribute
        sum f64, min T, max T, avg f64."""
        b = self.res[0] * self.res[1]
        t = self.x.dtype.itemsize
        return b * (8 + len(self.attrs) * (8 + 8 + 2 * t))


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _plummer_xy(rng: np.random.Generator, n: int, a: float = 1.0, rmax: float = 10.0):
    """3D Plummer positions (scale radius a, truncated at rmax); returns x, y, z.

    The enclosed-mass fraction is M(r) = r^3 / (r^2 + a^2)^(3/2); drawing
    u ~ U(0, M(rmax)] and inverting gives r = a / sqrt(u^(-2/3) - 1).
    Directions are isotropic.
    """
    m_max = rmax ** 3 / (rmax ** 2 + a ** 2) ** 1.5
    u = m_max * (1.0 - rng.random(n))  # (0, M(rmax)]
    r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    del u
    cos_t = rng.uniform(-1.0, 1.0, n)
    sin_t = np.sqrt(np.maximum(0.0, 1.0 - cos_t * cos_t))
    phi = rng.uniform(0.0, 2.0 * math.pi, n)
    x = r * sin_t * np.cos(phi)
    y = r * sin_t * np.sin(phi)
    z = r * cos_t
    return x, y, z


def uniform(n: int = 100_000, seed: int = 0, dtype=np.float64, res: int = 64) -> Workload:
    """x, y ~ U[0,1)^2; attributes mass ~ U[1,2] and speed ~ |N(0,1)|;
    a res x res grid over [0,1)^2."""
    rng = _rng(seed)
    x = rng.random(n)
    y = rng.random(n)
    mass = rng.uniform(1.0, 2.0, n)
    speed = np.abs(rng.standard_normal(n))
    cols = [np.ascontiguousarray(c, dtype=dtype) for c in (x, y, mass, speed)]
    return Workload(f"uniform n={n} {np.dtype(dtype).name} {res}x{res}",
                    cols[0], cols[1], cols[2:], (0.0, 0.0), (1.0, 1.0), (res, res))


def plummer(n: int = 50_000_000, seed: int = 0, dtype=np.float64, res: int = 1024,
            n_attrs: int = 3) -> Workload:
    """Plummer sphere (a = 1, truncated at r = 10) projected onto x-y;
    attributes mass ~ U[1,2], vx ~ N(0,1), vy ~ N(0,1) (the first n_attrs);
    a res x res grid over [-10,10]^2. z is drawn but not returned."""
    rng = _rng(seed)
    x, y, _z = _plummer_xy(rng, n)
    del _z
    attrs = [rng.uniform(1.0, 2.0, n), rng.standard_normal(n), rng.standard_normal(n)][:n_attrs]
    x = np.ascontiguousarray(x, dtype=dtype)
    y = np.ascontiguousarray(y, dtype=dtype)
    attrs = [np.ascontiguousarray(a, dtype=dtype) for a in attrs]
    return Workload(f"plummer n={n} {np.dtype(dtype).name} {res}x{res}",
                    x, y, attrs, (-10.0, -10.0), (10.0, 10.0), (res, res))


def gaussians(n: int = 2 ** 27, seed: int = 0, dtype=np.float32, res: int = 4096,
              n_comp: int = 16) -> Workload:
    """Mixture of n_comp isotropic Gaussians: centres ~ U[0,1)^2, sigma
    log-uniform in [1e-3, 5e-2], component chosen uniformly per particle;
    2 attributes ~ U[0, 1e4]; a res x res grid over [0,1)^2."""
    rng = _rng(seed)
    centres = rng.random((n_comp, 2))
    sigma = np.exp(rng.uniform(math.log(1e-3), math.log(5e-2), n_comp))
    comp = rng.integers(0, n_comp, n)
    x = centres[comp, 0] + sigma[comp] * rng.standard_normal(n)
    y = centres[comp, 1] + sigma[comp] * rng.standard_normal(n)
    del comp
    a0 = rng.uniform(0.0, 1e4, n)
    a1 = rng.uniform(0.0, 1e4, n)
    cols = [np.ascontiguousarray(c, dtype=dtype) for c in (x, y, a0, a1)]
    return Workload(f"gaussians n={n} {np.dtype(dtype).name} {res}x{res}",
                    cols[0], cols[1], cols[2:], (0.0, 0.0), (1.0, 1.0), (res, res))


# The 9 coordinate systems of the fused multi-grid workload: three position
# planes, three velocity planes and three position-velocity pairs.
PHASE_SPACE_SYSTEMS = [("x", "y"), ("x", "z"), ("y", "z"), ("vx", "vy"), ("vx", "vz"), ("vy", "vz"),
                       ("x", "vx"), ("y", "vy"), ("z", "vz")]
# The 10 variables binned in every system.
PHASE_SPACE_VARIABLES = ["mass", "vx", "vy", "vz", "speed", "ke", "r", "phi", "lz", "ly"]
PHASE_SPACE_BOUNDS = {"x": 10.0, "y": 10.0, "z": 10.0, "vx": 4.0, "vy": 4.0, "vz": 4.0}


def phase_space(n: int = 2 ** 22, seed: int = 0, dtype=np.float64):
    """An N-body snapshot for the fused multi-grid workload (the in situ
    step of Sec. 4.3: 10 variables binned in 9 coordinate systems). Plummer
    positions (a = 1, r < 10) in 3D, isotropic N(0,1) velocities, mass
    U[1,2], and derived scalars: speed, kinetic energy, radius, a softened
    potential -m / sqrt(r^2 + 1), and angular momenta lz = x vy - y vx,
    ly = z vx - x vz. Returns a dict name -> column."""
    rng = _rng(seed)
    x, y, z = _plummer_xy(rng, n)
    vx, vy, vz = rng.standard_normal((3, n))
    mass = rng.uniform(1.0, 2.0, n)
    speed = np.sqrt(vx * vx + vy * vy + vz * vz)
    r = np.sqrt(x * x + y * y + z * z)
    cols = {"x": x, "y": y, "z": z, "vx": vx, "vy": vy, "vz": vz, "mass": mass, "speed": speed,
            "ke": 0.5 * mass * speed * speed, "r": r, "phi": -mass / np.sqrt(r * r + 1.0),
            "lz": x * vy - y * vx, "ly": z * vx - x * vz}
    return {k: np.ascontiguousarray(v, dtype=dtype) for k, v in cols.items()}


@dataclasses.dataclass
class BatchPlan:
    """Per-block parameters of a batch; ``block(k)`` draws block k's data."""

    seed: int
    sizes: np.ndarray
    kinds: np.ndarray      # 0 = uniform over [0,1)^2, 1 = Plummer over [-10,10]^2
    sides: np.ndarray
    dtype: np.dtype
    child_seeds: Sequence

    @property
    def n_blocks(self) -> int:
        return int(self.sizes.shape[0])

    def block(self, k: int) -> Workload:
        n = int(self.sizes[k])
        side = int(self.sides[k])
        rng = np.random.Generator(np.random.PCG64(self.child_seeds[k]))
        if self.kinds[k] == 0:
            x = rng.random(n)
            y = rng.random(n)
            lo, hi = (0.0, 0.0), (1.0, 1.0)
        else:
            x, y, _ = _plummer_xy(rng, n)
            lo, hi = (-10.0, -10.0), (10.0, 10.0)
        mass = rng.uniform(1.0, 2.0, n)
        speed = np.abs(rng.standard_normal(n))
        cols = [np.ascontiguousarray(c, dtype=self.dtype) for c in (x, y, mass, speed)]
        kind = "uniform" if self.kinds[k] == 0 else "plummer"
        return Workload(f"block{k} {kind} n={n} {side}x{side}", cols[0], cols[1], cols[2:],
                        lo, hi, (side, side))

    def blocks(self) -> List[Workload]:
        return [self.block(k) for k in range(self.n_blocks)]


def batch(n_blocks: int = 256, seed: int = 0, dtype=np.float32,
          size_range=(1e3, 1e7), side_range=(32, 2048)) -> BatchPlan:
    """n_blocks uneven blocks: size log-uniform in size_range, kind uniform
    or Plummer by a fair coin, square grid side log-uniform in side_range."""
    rng = _rng(seed)
    sizes = np.floor(np.exp(rng.uniform(math.log(size_range[0]), math.log(size_range[1]),
                                        n_blocks))).astype(np.int64)
    kinds = rng.integers(0, 2, n_blocks)
    sides = np.floor(np.exp(rng.uniform(math.log(side_range[0]), math.log(side_range[1]),
                                        n_blocks))).astype(np.int64)
    children = np.random.SeedSequence(seed).spawn(n_blocks)
    return BatchPlan(seed, sizes, kinds, sides, np.dtype(dtype), children)


@dataclasses.dataclass
class ServingPlan:
    """A Poisson request stream over one particle pool (Plummer, f32)."""

    pool: Workload
    arrival_s: np.ndarray   # arrival time of each request, seconds from start
    sizes: np.ndarray
    offsets: np.ndarray     # request i bins pool[offsets[i] : offsets[i] + sizes[i]]
    sides: np.ndarray

    @property
    def n_requests(self) -> int:
        return int(self.sizes.shape[0])


def serving(n_requests: int = 10_000, seed: int = 0, mean_gap_s: float = 2e-3,
            size_range=(1e4, 2e7), side_range=(64, 1024), pool_n: Optional[int] = None,
            dtype=np.float32) -> ServingPlan:
    """Arrivals with Exp(mean_gap_s) gaps; size and grid side log-uniform;
    each request is a sub-range of a Plummer pool binned over [-10,10]^2."""
    rng = _rng(seed)
    gaps = rng.exponential(mean_gap_s, n_requests)
    arrival = np.cumsum(gaps) - gaps[0]
    sizes = np.floor(np.exp(rng.uniform(math.log(size_range[0]), math.log(size_range[1]),
                                        n_requests))).astype(np.int64)
    sides = np.floor(np.exp(rng.uniform(math.log(side_range[0]), math.log(side_range[1]),
                                        n_requests))).astype(np.int64)
    if pool_n is None:
        pool_n = int(sizes.max())
    pool_n = max(pool_n, int(sizes.max()))
    offsets = (rng.random(n_requests) * (pool_n - sizes + 1)).astype(np.int64)
    pool = plummer(pool_n, seed=seed + 1, dtype=dtype, res=1024, n_attrs=3)
    pool.attrs[2] = np.abs(pool.attrs[2])
    return ServingPlan(pool, arrival, sizes, offsets, sides)


def named(name: str, seed: int = 0, scale: float = 1.0):
    """The five workloads at full size (scale = 1) or scaled down in N."""
    def sz(n):
        return max(1, int(round(n * scale)))
    if name == "uniform64":
        return uniform(sz(100_000), seed)
    if name == "uniform64_at_scale":
        return uniform(sz(2 ** 27), seed)
    if name == "plummer1024":
        return plummer(sz(50_000_000), seed)
    if name == "gaussians4096":
        return gaussians(sz(2 ** 27), seed)
    raise KeyError(name)
