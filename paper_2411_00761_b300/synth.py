"""Seeded synthetic particle frames shaped like the paper's workloads.

This module holds no compression arithmetic: it only draws inputs, and both
the CUDA path and the CPU oracle consume what it returns.  The paper's own
datasets (HACC, WarpX, Copper, Helium, LJ, YIIP, 3DEP, BUN-ZIPPER; Table 1)
are not available, so these generators stand in for them:

* ``uniform_clusters`` -- plain LCP-S frame: 90% uniform in [0,1)^3, 10% from
  64 Gaussian clusters (sigma 0.01).
* ``md_fcc`` -- MD-like frame: FCC lattice (4 sites per cubic cell, lattice
  constant 1.0) with Gaussian thermal displacement; a seeded random subset of
  sites when fewer particles than sites are asked for.
* ``cosmology`` -- HACC-like frame with 6 fields (x, y, z, vx, vy, vz): 70% of
  particles in halos with an r^-2 density profile (so the enclosed mass grows
  linearly and r ~ U(0, r_vir)), 30% uniform background, periodic box,
  velocities N(0, 300^2) plus a per-halo bulk flow N(0, 300^2).
* ``brownian_trajectory`` -- multi-frame MD trajectory: FCC start, independent
  Gaussian steps per frame.

All frames are float32, field-major ([D, N], "SoA"), and particles are in a
seeded random storage order (storage order is unrelated to space, as in the
paper's discussion of particle storage order).
"""
from __future__ import annotations

import math

import numpy as np

FCC_BASIS = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])


def uniform_clusters(n: int = 1 << 20, seed: int = 0, n_clusters: int = 64,
                     sigma: float = 0.01, cluster_frac: float = 0.10) -> np.ndarray:
    """xyz [3, n]: uniform in [0,1)^3 plus Gaussian clusters (no clipping)."""
    rng = np.random.default_rng(seed)
    n_cl = int(round(n * cluster_frac))
    centers = rng.random((n_clusters, 3))
    which = rng.integers(0, n_clusters, size=n_cl)
    cl = centers[which] + rng.normal(0.0, sigma, size=(n_cl, 3))
    un = rng.random((n - n_cl, 3))
    pts = np.concatenate([un, cl], axis=0)
    pts = pts[rng.permutation(n)]
    return np.ascontiguousarray(pts.T.astype(np.float32))


def _fcc_sites(idx: np.ndarray, cells: int) -> np.ndarray:
    cell, basis = np.divmod(idx, 4)
    cx = cell % cells
    cy = (cell // cells) % cells
    cz = cell // (cells * cells)
    return np.stack([cx, cy, cz], axis=1).astype(np.float64) + FCC_BASIS[basis]


def md_fcc(n: int = 1 << 24, seed: int = 1, cells: int = 252, lattice: float = 1.0,
           sigma: float = 0.05) -> np.ndarray:
    """xyz [3, n] on an FCC lattice of cells^3 cubic cells plus N(0, sigma^2)."""
    rng = np.random.default_rng(seed)
    n_sites = 4 * cells ** 3
    if n > n_sites:
        raise ValueError("more particles than lattice sites")
    idx = rng.permutation(n_sites)[:n] if n < n_sites else rng.permutation(n_sites)
    out = np.empty((3, n), dtype=np.float32)
    step = 1 << 22
    for s in range(0, n, step):
        e = min(n, s + step)
        pos = _fcc_sites(idx[s:e], cells) * lattice
        pos += rng.normal(0.0, sigma, size=pos.shape)
        out[:, s:e] = pos.T
    return out


def cosmology(n: int = 1 << 26, seed: int = 2, box: float = 1000.0, n_halos: int = 4096,
              halo_frac: float = 0.70, sigma_v: float = 300.0) -> np.ndarray:
    """[6, n]: positions in a periodic box and velocities (x, y, z, vx, vy, vz)."""
    rng = np.random.default_rng(seed)
    centers = rng.random((n_halos, 3)) * box
    r_vir = rng.uniform(0.5, 3.0, size=n_halos)
    bulk = rng.normal(0.0, sigma_v, size=(n_halos, 3))
    is_halo = rng.random(n) < halo_frac
    halo_of = rng.integers(0, n_halos, size=n)
    out = np.empty((6, n), dtype=np.float32)
    step = 1 << 22
    for s in range(0, n, step):
        e = min(n, s + step)
        m = e - s
        h = halo_of[s:e]
        inh = is_halo[s:e]
        # halo members: r ~ U(0, r_vir) (r^-2 density), isotropic direction
        u = rng.normal(size=(m, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        r = rng.random(m) * r_vir[h]
        pos_h = centers[h] + u * r[:, None]
        pos_b = rng.random((m, 3)) * box
        pos = np.where(inh[:, None], pos_h, pos_b)
        pos = np.mod(pos, box)
        pos[pos >= box] = 0.0  # float rounding of the wrap
        vel = rng.normal(0.0, sigma_v, size=(m, 3)) + np.where(inh[:, None], bulk[h], 0.0)
        out[0:3, s:e] = pos.T
        out[3:6, s:e] = vel.T
    return out


def fcc_block_start(n: int, lattice: float = 1.0) -> np.ndarray:
    """First n sites of the smallest cubic FCC block holding at least n sites,
    as [3, n] float64."""
    cells = max(1, math.ceil((n / 4) ** (1.0 / 3.0)))
    while 4 * cells ** 3 < n:
        cells += 1
    return (_fcc_sites(np.arange(n), cells) * lattice).T.copy()


def brownian_trajectory(n: int, n_frames: int, seed: int, sigma: float = 0.02,
                        lattice: float = 1.0):
    """Yields n_frames frames [3, n] (float32) of a Brownian trajectory that
    starts on an FCC block; particle i keeps storage slot i in every frame."""
    rng = np.random.default_rng(seed)
    order = rng.permutation(n)
    pos = fcc_block_start(n, lattice)[:, order]
    for _ in range(n_frames):
        yield np.ascontiguousarray(pos.astype(np.float32))
        pos = pos + rng.normal(0.0, sigma, size=pos.shape)


def trajectory_sizes(n_traj: int = 64, lo: float = 1e4, hi: float = 4e6, seed: int = 3) -> list[int]:
    """Log-uniform particle counts of the multi-frame workload."""
    rng = np.random.default_rng(seed)
    return [int(round(math.exp(v))) for v in rng.uniform(math.log(lo), math.log(hi), size=n_traj)]


def serving_requests(n_req: int, seed: int = 4, n_producers: int = 64, rate: float = 2000.0,
                     n_lo: float = 1e4, n_hi: float = 8e6, eb_lo: float = 1e-5,
                     eb_hi: float = 1e-2) -> list[dict]:
    """Request descriptors of the serving workload: Poisson arrivals over
    n_producers streams at an aggregate rate, log-uniform sizes and relative
    error bounds, generator kind drawn from the three single-frame shapes,
    and a 50/50 compress/decompress mix (a decompress replays an earlier
    output of the same stream)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    out = []
    for i in range(n_req):
        out.append(dict(
            t=float(t[i]),
            producer=int(rng.integers(0, n_producers)),
            n=int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))))),
            eb=float(math.exp(rng.uniform(math.log(eb_lo), math.log(eb_hi)))),
            kind=int(rng.integers(0, 3)),
            op="compress" if rng.random() < 0.5 else "decompress",
            seed=int(rng.integers(0, 2 ** 31)),
        ))
    return out


def frame_for_request(kind: int, n: int, seed: int) -> np.ndarray:
    """xyz [3, n] drawn from one of the three single-frame generators."""
    if kind == 0:
        return uniform_clusters(n, seed)
    if kind == 1:
        cells = max(1, math.ceil((n / 4) ** (1.0 / 3.0)) + 1)
        return md_fcc(n, seed, cells=cells)
    return np.ascontiguousarray(cosmology(n, seed)[0:3])
