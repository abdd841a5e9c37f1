"""Seeded synthetic particle sets for the adaptive 3-D Laplace FMM.

This module only draws inputs.  It holds none of the method's arithmetic
(no keys, no trees, no expansions), so both the CPU oracle and the CUDA
path can take their inputs from it without sharing any computation.

Random numbers come from Philox4x32-10, the counter-based generator of
Salmon, Moraes, Dror and Shaw ("Parallel random numbers: as easy as 1, 2, 3",
SC'11), written here from that definition.  A stream is the key (two 32-bit
words from the seed) plus a stream id in counter word 1; counter word 0 walks
the draws.  Every value depends only on (seed, stream, index), so results are
identical on every machine and numpy version.

Distributions (the paper's workload is particles spread at random in a unit
cube, Section 5; the irregular sets exercise the adaptive octree of
Section 2.1):

* ``uniform``   -- uniform in [0,1)^3.
* ``plummer``   -- Plummer sphere, scale radius ``a``: r = a (u^(-2/3) - 1)^(-1/2),
                   redrawn while r > ``rmax``; isotropic direction (z ~ U[-1,1],
                   azimuth ~ U[0, 2 pi)).
* ``clustered`` -- ``nclusters`` centres uniform in [0,1)^3; particle i belongs to
                   cluster i mod nclusters and is offset by N(0, sigma^2) per axis.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "philox4x32_10", "Stream", "uniform_cube", "plummer", "clustered",
    "charges_uniform", "charges_normal", "charges_constant", "Workload",
    "make_workload", "WORKLOADS", "batched_sizes",
]

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: tuple[int, int]) -> np.ndarray:
    """Philox4x32 with 10 rounds.  ``ctr`` is (n, 4) uint32; returns (n, 4) uint32."""
    c = np.asarray(ctr, dtype=np.uint64).copy()
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & 0xFFFFFFFF
            k1 = (k1 + _W1) & 0xFFFFFFFF
        p0 = _M0 * c[:, 0]
        p1 = _M1 * c[:, 2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        n0 = hi1 ^ c[:, 1] ^ np.uint64(k0)
        n2 = hi0 ^ c[:, 3] ^ np.uint64(k1)
        c[:, 0], c[:, 1], c[:, 2], c[:, 3] = n0, lo1, n2, lo0
    return c.astype(np.uint32)


class Stream:
    """Sequential draws from one Philox stream (seed, stream id)."""

    def __init__(self, seed: int, stream: int = 0):
        self.key = (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
        self.stream = stream & 0xFFFFFFFF
        self.pos = 0  # next counter value (each counter yields two doubles)

    def _blocks(self, nblocks: int) -> np.ndarray:
        idx = np.arange(self.pos, self.pos + nblocks, dtype=np.uint64)
        self.pos += nblocks
        ctr = np.zeros((nblocks, 4), dtype=np.uint64)
        ctr[:, 0] = idx & _MASK32
        ctr[:, 1] = np.uint64(self.stream)
        ctr[:, 2] = idx >> np.uint64(32)
        return philox4x32_10(ctr, self.key)

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1) with 53 random bits each."""
        nb = (n + 1) // 2
        w = self._blocks(nb).astype(np.uint64)
        a = np.empty(2 * nb, dtype=np.uint64)
        b = np.empty(2 * nb, dtype=np.uint64)
        a[0::2], b[0::2] = w[:, 0] >> np.uint64(5), w[:, 1] >> np.uint64(6)
        a[1::2], b[1::2] = w[:, 2] >> np.uint64(5), w[:, 3] >> np.uint64(6)
        u = (a * np.uint64(1 << 26) + b).astype(np.float64) * (1.0 / 9007199254740992.0)
        return u[:n]

    def normal(self, n: int) -> np.ndarray:
        """n standard normals by the Box-Muller transform."""
        m = (n + 1) // 2
        u1 = 1.0 - self.uniform(m)  # (0, 1]
        u2 = self.uniform(m)
        rad = np.sqrt(-2.0 * np.log(u1))
        z = np.empty(2 * m)
        z[0::2] = rad * np.cos(2.0 * math.pi * u2)
        z[1::2] = rad * np.sin(2.0 * math.pi * u2)
        return z[:n]


def uniform_cube(n: int, rng: Stream) -> np.ndarray:
    return rng.uniform(3 * n).reshape(n, 3)


def plummer(n: int, rng: Stream, a: float = 1.0, rmax: float = 50.0) -> np.ndarray:
    """Plummer sphere of scale radius ``a``, truncated by redrawing at r > rmax."""
    radii = np.empty(0)
    while radii.size < n:
        need = n - radii.size
        u = 1.0 - rng.uniform(need + need // 8 + 16)  # (0, 1]
        with np.errstate(divide="ignore"):
            r = a / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
        r = r[np.isfinite(r) & (r <= rmax)]
        radii = np.concatenate([radii, r])
    radii = radii[:n]
    z = 2.0 * rng.uniform(n) - 1.0
    az = 2.0 * math.pi * rng.uniform(n)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([radii * s * np.cos(az), radii * s * np.sin(az), radii * z], axis=1)


def clustered(n: int, rng: Stream, nclusters: int = 64, sigma: float = 0.01) -> np.ndarray:
    centres = rng.uniform(3 * nclusters).reshape(nclusters, 3)
    off = sigma * rng.normal(3 * n).reshape(n, 3)
    return centres[np.arange(n) % nclusters] + off


def charges_uniform(n: int, rng: Stream) -> np.ndarray:
    return 2.0 * rng.uniform(n) - 1.0


def charges_normal(n: int, rng: Stream) -> np.ndarray:
    return rng.normal(n)


def charges_constant(n: int, value: float) -> np.ndarray:
    return np.full(n, value)


@dataclass
class Workload:
    """One synthetic system plus the FMM parameters it is run with."""
    name: str
    pos: np.ndarray            # (n, 3) float64
    q: np.ndarray              # (n,) float64
    p: int
    leaf_size: int
    theta: float
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.pos.shape[0])


def _dist(kind: str, n: int, rng: Stream) -> np.ndarray:
    if kind == "uniform":
        return uniform_cube(n, rng)
    if kind == "plummer":
        return plummer(n, rng)
    if kind == "clustered":
        return clustered(n, rng)
    raise ValueError(kind)


# name -> (config number, distribution, default n, charges, p, leaf, theta)
WORKLOADS = {
    "uniform": (1, "uniform", 16384, "uniform", 4, 64, 0.5),
    "plummer": (2, "plummer", 1 << 20, "one_over_n", 8, 64, 0.4),
    "clustered": (3, "clustered", 1 << 22, "uniform", 10, 64, 0.5),
    "gradient": (4, "uniform", 1 << 20, "normal", 8, 64, 0.5),
}


def make_workload(name: str, n: int | None = None, seed: int | None = None) -> Workload:
    """Build a named workload; ``n`` overrides the particle count (same recipe)."""
    cfg, kind, n0, qkind, p, leaf, theta = WORKLOADS[name]
    n = n0 if n is None else int(n)
    seed = 12030889 * 10 + cfg if seed is None else int(seed)
    rng_x = Stream(seed, 0)
    rng_q = Stream(seed, 1)
    pos = _dist(kind, n, rng_x)
    if qkind == "uniform":
        q = charges_uniform(n, rng_q)
    elif qkind == "normal":
        q = charges_normal(n, rng_q)
    else:
        q = charges_constant(n, 1.0 / max(n, 1))
    extra = {}
    if name == "gradient":
        extra["w"] = Stream(seed, 2).normal(n)
    return Workload(name, pos, q, p, leaf, theta, extra)


def batched_sizes(nsys: int = 512, lo: int = 1024, hi: int = 65536, seed: int | None = None) -> np.ndarray:
    """System sizes floor(exp(U[ln lo, ln hi])) for the batched workload."""
    seed = 12030889 * 10 + 5 if seed is None else seed
    u = Stream(seed, 7).uniform(nsys)
    return np.floor(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def make_batched(nsys: int = 512, seed: int | None = None, sizes: np.ndarray | None = None):
    """Systems alternating uniform / Plummer / clustered, charges U[-1,1]."""
    seed = 12030889 * 10 + 5 if seed is None else seed
    if sizes is None:
        sizes = batched_sizes(nsys, seed=seed)
    kinds = ("uniform", "plummer", "clustered")
    out = []
    for s, ns in enumerate(sizes):
        rx, rq = Stream(seed, 16 + 2 * s), Stream(seed, 17 + 2 * s)
        out.append((_dist(kinds[s % 3], int(ns), rx), charges_uniform(int(ns), rq)))
    return out
