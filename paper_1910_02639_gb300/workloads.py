"""Seeded synthetic particle sets for the b-tree neighbour search.

Input recipes only: this module holds none of the method's arithmetic (no tree,
no distance predicate, no kernel).  Both the CUDA path and the CPU oracle are
fed from here.  All generators use numpy's PCG64 with an explicit seed, so a
seed names one input exactly.  Positions and smoothing lengths are float32;
masses are float32 (1/N unless stated).

Workloads (the paper's EC and SP datasets of Sec. 4.1 are not available; these
synthetic sets take their sizes and character):
  uniform_cube     -- N points uniform in [0,1)^3, one h so that the 2h sphere
                      holds ~T expected neighbours (small plain case).
  evrard           -- Evrard-like collapse: radius r = R sqrt(u) (density
                      ~ 1/r), isotropic directions; h_i from the local density
                      n(r) = N / (2 pi R^2 r) so that the 2h sphere holds ~100.
  jittered_slab    -- nx*ny*nz cubic lattice, spacing 1, uniform jitter
                      +-0.1 per coordinate, h = 1.5 (SP-like, near uniform).
  lattice          -- the same lattice with no jitter (closed-form counts).
  plummer          -- Plummer sphere of scale a, truncated at 20 a.
  batched_sets     -- many independent sets, sizes log-uniform, each from
                      uniform-cube / 1/r-sphere / Plummer, T ~ U[50,150].
  request_stream   -- Poisson arrivals of jobs with log-uniform sizes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class ParticleSet:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    h: np.ndarray
    m: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def positions(self) -> np.ndarray:
        return np.stack([self.x, self.y, self.z], axis=1)


def _pack(x, y, z, h, m=None, name="", **meta) -> ParticleSet:
    n = x.shape[0]
    if m is None:
        m = np.full(n, 1.0 / max(n, 1), np.float32)
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return ParticleSet(f(x), f(y), f(z), f(h), f(m), name, dict(meta))


def _h_for_target(target: float, number_density):
    """h such that the 2h sphere holds `target` expected particles."""
    return 0.5 * np.cbrt(3.0 * target / (4.0 * math.pi * number_density))


def uniform_cube(n: int = 32768, seed: int = 1911, target: float = 100.0) -> ParticleSet:
    rng = np.random.Generator(np.random.PCG64(seed))
    p = rng.random((3, n), dtype=np.float32)
    h = np.full(n, np.float32(_h_for_target(target, float(n))), np.float32)
    return _pack(p[0], p[1], p[2], h, name="uniform_cube", seed=seed, target=target)


def evrard(n: int = 1_000_000, seed: int = 1912, radius: float = 1.0,
           target: float = 100.0) -> ParticleSet:
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random(n)
    r = radius * np.sqrt(u)
    d = rng.standard_normal((3, n))
    d /= np.sqrt((d * d).sum(axis=0))
    pos = (d * r).astype(np.float32)
    rr = np.maximum(np.sqrt((pos.astype(np.float64) ** 2).sum(axis=0)), 1e-12)
    dens = n / (2.0 * math.pi * radius * radius * rr)
    h = _h_for_target(target, dens).astype(np.float32)
    return _pack(pos[0], pos[1], pos[2], h, name="evrard", seed=seed, target=target)


def jittered_slab(nx: int = 400, ny: int = 250, nz: int = 100, jitter: float = 0.1,
                  h: float = 1.5, seed: int = 1913) -> ParticleSet:
    """Lattice points (i, j, k), x fastest, each coordinate + U(-jitter, jitter)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = nx * ny * nz
    ix = np.arange(n, dtype=np.int64)
    x = (ix % nx).astype(np.float32)
    y = ((ix // nx) % ny).astype(np.float32)
    z = (ix // (nx * ny)).astype(np.float32)
    if jitter > 0:
        j = rng.uniform(-jitter, jitter, size=(3, n)).astype(np.float32)
        x, y, z = x + j[0], y + j[1], z + j[2]
    hh = np.full(n, np.float32(h), np.float32)
    return _pack(x, y, z, hh, name="jittered_slab", seed=seed, nx=nx, ny=ny, nz=nz,
                 jitter=jitter)


def lattice(nx: int, ny: int, nz: int, h: float = 1.5) -> ParticleSet:
    return jittered_slab(nx, ny, nz, jitter=0.0, h=h, seed=0)


def plummer(n: int, seed: int, scale: float = 0.1, truncate: float = 20.0,
            target: float = 100.0) -> ParticleSet:
    """Plummer sphere: M(<r)/M = r^3/(r^2+a^2)^(3/2); samples beyond
    truncate*a are redrawn."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rmax = truncate * scale
    mmax = rmax ** 3 / (rmax ** 2 + scale ** 2) ** 1.5
    u = rng.random(n) * mmax
    r = scale / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    d = rng.standard_normal((3, n))
    d /= np.sqrt((d * d).sum(axis=0))
    pos = (d * r).astype(np.float32)
    rr = np.sqrt((pos.astype(np.float64) ** 2).sum(axis=0))
    dens = (n / mmax) * 3.0 / (4.0 * math.pi * scale ** 3) * (1.0 + (rr / scale) ** 2) ** -2.5
    h = _h_for_target(target, dens).astype(np.float32)
    return _pack(pos[0], pos[1], pos[2], h, name="plummer", seed=seed, scale=scale,
                 target=target)


def sphere_1r(n: int, seed: int, radius: float = 1.0, target: float = 100.0) -> ParticleSet:
    s = evrard(n, seed=seed, radius=radius, target=target)
    s.name = "sphere_1r"
    return s


def cube(n: int, seed: int, target: float = 100.0) -> ParticleSet:
    return uniform_cube(n, seed=seed, target=target)


KINDS = ("uniform_cube", "sphere_1r", "plummer")


def make_set(kind: str, n: int, seed: int, target: float) -> ParticleSet:
    if kind == "uniform_cube":
        return cube(n, seed, target)
    if kind == "sphere_1r":
        return sphere_1r(n, seed, target=target)
    if kind == "plummer":
        return plummer(n, seed, target=target)
    raise ValueError(kind)


def batched_specs(nsets: int = 256, seed: int = 1914, nmin: float = 1e3,
                  nmax: float = 1e6):
    """(kind, n, seed, target) of each set of the batched workload."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = np.exp(rng.uniform(math.log(nmin), math.log(nmax), nsets)).astype(np.int64)
    kinds = rng.integers(0, len(KINDS), nsets)
    targets = rng.uniform(50.0, 150.0, nsets)
    seeds = rng.integers(0, 2 ** 31 - 1, nsets)
    return [(KINDS[int(k)], int(n), int(s), float(t))
            for k, n, s, t in zip(kinds, ns, seeds, targets)]


def batched_sets(nsets: int = 256, seed: int = 1914, nmin: float = 1e3,
                 nmax: float = 1e6):
    return [make_set(*spec) for spec in batched_specs(nsets, seed, nmin, nmax)]


def request_stream(nreq: int, seed: int = 1915, rate: float = 200.0,
                   nmin: float = 1e4, nmax: float = 2e6):
    """Poisson arrivals: list of (arrival_time_s, kind, n, seed, target)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, nreq))
    ns = np.exp(rng.uniform(math.log(nmin), math.log(nmax), nreq)).astype(np.int64)
    kinds = rng.integers(0, len(KINDS), nreq)
    targets = rng.uniform(50.0, 150.0, nreq)
    seeds = rng.integers(0, 2 ** 31 - 1, nreq)
    return [(float(a), KINDS[int(k)], int(n), int(s), float(tg))
            for a, k, n, s, tg in zip(t, kinds, ns, seeds, targets)]
