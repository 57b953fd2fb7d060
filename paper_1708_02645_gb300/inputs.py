"""Seeded synthetic inputs for the B-spline orbital workloads.

This module holds input recipes only: random coefficient tables, plane-wave
orbitals sampled on the grid, electron positions and walker sizes.  It holds
none of the B-spline arithmetic, so both the CUDA path and the FP64 oracle
can be fed from it without sharing any of the method's code.

Randomness comes from a counter-based splitmix64 stream (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), so the
same seed gives the same bits on any host and any numpy version.

The DFT orbitals of the paper's NiO benchmarks (Table 1) are not available,
so plane-wave orbitals with the NiO supercells' shapes stand in for them:
each orbital is the real part of 8 plane waves with integer wave vectors
|k| <= 4 and complex Gaussian amplitudes, sampled on the grid nodes and used
directly as B-spline coefficients.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
SEED_BASE = 20170808


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n outputs of splitmix64 from state seed, counters offset .. offset+n-1."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n doubles uniform in [0, 1) (53-bit)."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int) -> np.ndarray:
    """n standard normal doubles (Box-Muller on two uniform streams)."""
    m = (n + 1) // 2
    u1 = uniform01(seed, m, 0)
    u2 = uniform01(seed, m, m)
    r = np.sqrt(-2.0 * np.log1p(-u1))  # 1 - u1 in (0, 1]
    z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])
    return z[:n]


def uniform_coefs(nx: int, ny: int, nz: int, N: int, seed: int) -> np.ndarray:
    """Coefficient table [nx, ny, nz, N] with i.i.d. U(-1, 1) entries, FP64."""
    u = uniform01(seed, nx * ny * nz * N)
    return (2.0 * u - 1.0).reshape(nx, ny, nz, N)


def wavevectors(kmax: float = 4.0) -> np.ndarray:
    """All integer k in Z^3 with Euclidean |k| <= kmax, lexicographic order."""
    r = int(math.floor(kmax))
    ks = [(a, b, c) for a in range(-r, r + 1) for b in range(-r, r + 1)
          for c in range(-r, r + 1) if a * a + b * b + c * c <= kmax * kmax + 1e-9]
    return np.asarray(ks, dtype=np.int64)


def plane_wave_spec(N: int, seed: int, kmax: float = 4.0, nwaves: int = 8):
    """Wave vectors k [N, nwaves, 3] (distinct per orbital, uniform without
    replacement) and amplitudes a [N, nwaves] = (g1 + i g2)/sqrt(2)."""
    kset = wavevectors(kmax)
    K = len(kset)
    keys = uniform01(seed, N * K).reshape(N, K)
    idx = np.argsort(keys, axis=1, kind="stable")[:, :nwaves]
    k = kset[idx]
    g = normal(seed + 1, 2 * N * nwaves).reshape(2, N, nwaves)
    a = (g[0] + 1j * g[1]) / math.sqrt(2.0)
    return k, a


def plane_wave_coefs(nx: int, ny: int, nz: int, N: int, seed: int,
                     kmax: float = 4.0, nwaves: int = 8,
                     dtype=np.float64) -> np.ndarray:
    """Coefficient table [nx, ny, nz, N]: orbital n sampled at node m as
    f_n(m/n) = Re sum_j a_nj exp(2 pi i k_nj . m/n)."""
    k, a = plane_wave_spec(N, seed, kmax, nwaves)
    out = np.empty((nx, ny, nz, N), dtype=dtype)
    mx, my, mz = np.arange(nx) / nx, np.arange(ny) / ny, np.arange(nz) / nz
    chunk = 16
    for n0 in range(0, N, chunk):
        n1 = min(N, n0 + chunk)
        kk = k[n0:n1]
        ex = np.exp(2j * np.pi * kk[:, :, 0, None] * mx)          # [n, J, nx]
        ey = np.exp(2j * np.pi * kk[:, :, 1, None] * my)          # [n, J, ny]
        ez = np.exp(2j * np.pi * kk[:, :, 2, None] * mz)          # [n, J, nz]
        A = a[n0:n1, :, None, None] * ex[:, :, :, None] * ey[:, :, None, :]  # [n,J,nx,ny]
        A = A.transpose(0, 2, 3, 1).reshape(n1 - n0, nx * ny, -1)  # [n, xy, J]
        F = np.matmul(A, ez).real                                  # [n, xy, nz]
        out[..., n0:n1] = F.reshape(n1 - n0, nx, ny, nz).transpose(1, 2, 3, 0)
    return out


def uniform_positions(P: int, seed: int) -> np.ndarray:
    """P positions [P, 3] uniform in the unit cube, FP32.  Each coordinate is
    a multiple of 2^-24, so it is exact in FP32 and strictly below 1."""
    bits = splitmix64(seed, 3 * P) >> np.uint64(40)
    return (bits.astype(np.float64) * (2.0 ** -24)).astype(np.float32).reshape(P, 3)


def wide_positions(P: int, seed: int, lo: float = -3.0, hi: float = 3.0) -> np.ndarray:
    """P positions [P, 3] uniform in [lo, hi)^3 (outside the unit cube, to
    exercise periodic wrap), rounded to FP32."""
    u = uniform01(seed, 3 * P)
    return (lo + (hi - lo) * u).astype(np.float32).reshape(P, 3)


def walker_sizes(nwalkers: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Electron counts per walker, uniform on the integers lo..hi inclusive."""
    u = uniform01(seed, nwalkers)
    return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64)


@dataclass(frozen=True)
class SplineConfig:
    """One synthetic orbital-set workload."""
    name: str
    grid: tuple
    N: int
    coefs: str            # "uniform" or "planewave"
    walkers: int
    per_walker: int
    seed: int
    dtypes: tuple = ("f32",)
    kinds: tuple = ("vgh",)
    note: str = ""

    @property
    def P(self) -> int:
        return self.walkers * self.per_walker

    def make_coefs(self, dtype=np.float64) -> np.ndarray:
        nx, ny, nz = self.grid
        if self.coefs == "uniform":
            return uniform_coefs(nx, ny, nz, self.N, self.seed).astype(dtype, copy=False)
        return plane_wave_coefs(nx, ny, nz, self.N, self.seed, dtype=dtype)

    def make_positions(self) -> np.ndarray:
        return uniform_positions(self.P, self.seed + 1000)


# Workloads.  Grid shapes follow the paper's NiO supercells scaled down from
# the 80^3 FFT grid of Table 1; N follows N/2 orbitals per spin for 384 and
# 768 electrons.
UNIFORM16 = SplineConfig("uniform16_n16", (16, 16, 16), 16, "uniform", 1, 1024,
                         SEED_BASE + 1, ("f64",), ("vgh",),
                         "i.i.d. U(-1,1) coefficients, FP64 table")
NIO32 = SplineConfig("nio32_48cubed_n192", (48, 48, 48), 192, "planewave", 32, 384,
                     SEED_BASE + 2, ("f32",), ("vgl", "vgh"),
                     "NiO-32 shape: 32 walkers x 384 electrons")
NIO64 = SplineConfig("nio64_64cubed_n384", (64, 64, 64), 384, "planewave", 128, 768,
                     SEED_BASE + 3, ("f32", "bf16", "f16"), ("vgh",),
                     "NiO-64 shape: 128 walkers x 768 electrons")

CONFIGS = {c.name: c for c in (UNIFORM16, NIO32, NIO64)}


@dataclass(frozen=True)
class CrowdConfig:
    """Several orbital sets and walkers of uneven size (batched launches)."""
    name: str = "crowd_3sets_512walkers"
    sets: tuple = ((32, 64), (48, 192), (64, 384))   # (grid edge, N)
    walkers: int = 512
    ne_lo: int = 64
    ne_hi: int = 768
    seed: int = SEED_BASE + 4

    def sizes(self) -> np.ndarray:
        return walker_sizes(self.walkers, self.ne_lo, self.ne_hi, self.seed)

    def set_of_walker(self) -> np.ndarray:
        """Walker w uses orbital set w mod (number of sets)."""
        return np.arange(self.walkers) % len(self.sets)

    def make_coefs(self, s: int, dtype=np.float64) -> np.ndarray:
        n, N = self.sets[s]
        return plane_wave_coefs(n, n, n, N, self.seed + 10 * (s + 1), dtype=dtype)

    def make_positions(self, w: int, ne: int) -> np.ndarray:
        return uniform_positions(int(ne), self.seed + 100000 + w)


CROWD = CrowdConfig()


def icosahedron_directions() -> np.ndarray:
    """The 12 unit vectors to the vertices of a regular icosahedron: the
    cyclic permutations of (0, +-1, +-g), g the golden ratio, normalised (the
    12-point rule for angular integrals over the sphere)."""
    g = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for s1 in (1.0, -1.0):
        for s2 in (1.0, -1.0):
            v += [(0.0, s1, s2 * g), (s1, s2 * g, 0.0), (s2 * g, 0.0, s1)]
    v = np.asarray(v)
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def random_rotations(seed: int, n: int) -> np.ndarray:
    """n rotation matrices [n, 3, 3], uniform on SO(3): unit quaternions from
    normalised 4-D Gaussian vectors."""
    q = normal(seed, 4 * n).reshape(n, 4)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], axis=1),
        np.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], axis=1),
        np.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], axis=1)], axis=1)


@dataclass(frozen=True)
class NlppConfig:
    """Quadrature points of the non-local pseudopotential for a batch of
    walkers (Sec. 3: an angular quadrature on a sphere around each ion, one
    determinant ratio per point).  Ions sit on an edge^3 lattice of the unit
    cube; every electron within r_cut of its nearest ion contributes the 12
    icosahedron points on the sphere through it about that ion, turned by a
    random rotation; each point's row of A^-1 is its electron's."""
    name: str = "nlpp_nio64_12pt"
    ion_edge: int = 4            # 64 ions, as in the 64-atom NiO cell
    r_cut: float = 0.09          # reduced units (about 1.5 bohr in a 16.7 bohr cell)
    walkers: int = 128
    electrons: int = 768
    seed: int = SEED_BASE + 5

    @property
    def n_electrons(self) -> int:
        return self.walkers * self.electrons

    def make_points(self):
        """(points [Q, 3] FP32 in [0, 1), row_of [Q] int32 electron index)."""
        e = uniform_positions(self.n_electrons, self.seed).astype(np.float64)
        a = float(self.ion_edge)
        ion = np.round(e * a) / a                 # nearest lattice site (periodic image)
        d = e - ion
        r = np.linalg.norm(d, axis=1)
        near = np.nonzero(r < self.r_cut)[0]
        rot = random_rotations(self.seed + 1, len(near))
        dirs = np.einsum("nij,kj->nki", rot, icosahedron_directions())      # [n, 12, 3]
        pts = ion[near, None, :] + r[near, None, None] * dirs
        pts = np.mod(pts, 1.0).reshape(-1, 3).astype(np.float32)
        pts[pts >= np.float32(1.0)] = np.float32(0.0)
        row_of = np.repeat(near.astype(np.int32), 12)
        return pts, row_of


NLPP = NlppConfig()
