"""Seeded synthetic inputs: LJ+ATM fluids in periodic boxes.

This module only draws positions and velocities; it holds none of the
method's arithmetic (no potentials, cells or traversals), so that the CPU
oracle and the CUDA path can both be fed from it.

The workloads follow the paper's homogeneous and slab scenarios (section 5):
fcc or uniform starts in cubic periodic boxes at a given reduced density,
Maxwell-Boltzmann velocities at a reduced temperature, and a liquid slab
surrounded by vapour.  All arrays are SoA float64 ``[3, n]``.  The seed of a
configuration is ``config_index * 1000 + replica``.
"""
import math

import numpy as np


def fcc_sites(m):
    """Unit-cube fcc lattice with m^3 cells (4 m^3 sites), coordinates in [0, 1)."""
    base = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    g = np.arange(m, dtype=np.float64)
    cx, cy, cz = np.meshgrid(g, g, g, indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    pts = (cells[:, None, :] + base[None, :, :]).reshape(-1, 3) / m
    return pts


def fcc_positions(n, box, rng, jitter=0.05):
    """n molecules on an fcc lattice filling a cubic box of edge ``box``.

    If n is not 4 m^3, the smallest lattice with at least n sites is used and
    a seeded random subset of n sites is kept.  Each coordinate gets a uniform
    jitter in [-jitter, +jitter]."""
    m = 1
    while 4 * m ** 3 < n:
        m += 1
    pts = fcc_sites(m) * box
    if pts.shape[0] > n:
        keep = np.sort(rng.choice(pts.shape[0], size=n, replace=False))
        pts = pts[keep]
    pts = pts + rng.uniform(-jitter, jitter, size=pts.shape)
    pts = np.mod(pts, box)
    return np.ascontiguousarray(pts.T)


def simple_cubic_positions(n, box, rng):
    """n molecules on a simple cubic lattice filling a cubic box of edge ``box``
    (the single-phase start of section 5.1); if n is not m^3, a seeded random
    subset of the smallest lattice with at least n sites is kept."""
    m = 1
    while m ** 3 < n:
        m += 1
    g = (np.arange(m, dtype=np.float64) + 0.5) * (box / m)
    cx, cy, cz = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
    if pts.shape[0] > n:
        pts = pts[np.sort(rng.choice(pts.shape[0], size=n, replace=False))]
    return np.ascontiguousarray(pts.T)


def uniform_positions(n, box, rng):
    box = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    return np.ascontiguousarray((rng.random((n, 3)) * box).T)


def maxwell_boltzmann(n, temperature, rng, exact=True):
    """Unit-mass velocities at reduced temperature T with zero net momentum.
    With ``exact`` the kinetic temperature 2K/(3n-3) is rescaled to T."""
    v = rng.normal(0.0, math.sqrt(temperature), size=(n, 3))
    v -= v.mean(axis=0, keepdims=True)
    if exact and n > 1:
        t = (v * v).sum() / (3 * n - 3)
        v *= math.sqrt(temperature / t)
    return np.ascontiguousarray(v.T)


def random_sequential(n_target, lo, hi, min_dist, rng, existing=None, box=None, max_tries=200):
    """Random sequential insertion of up to n_target points in the axis box
    [lo, hi) with a minimum (periodic, if ``box``) spacing; returns [k, 3]."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    pts = [] if existing is None else list(existing)
    md2 = min_dist * min_dist
    placed = 0
    arr = np.array(pts).reshape(-1, 3)
    for _ in range(n_target):
        for _try in range(max_tries):
            p = lo + rng.random(3) * (hi - lo)
            if arr.shape[0]:
                d = arr - p
                if box is not None:
                    d -= np.rint(d / box) * box
                if np.min((d * d).sum(axis=1)) < md2:
                    continue
            arr = np.vstack([arr, p[None, :]])
            placed += 1
            break
    return arr


def homogeneous(n, rho, temperature, seed, jitter=0.05):
    """Homogeneous liquid: fcc start in a cubic box at density rho."""
    rng = np.random.default_rng(seed)
    box = (n / rho) ** (1.0 / 3.0)
    x = fcc_positions(n, box, rng, jitter=jitter)
    v = maxwell_boltzmann(n, temperature, rng)
    return dict(x=x, v=v, box=np.array([box, box, box]), n=n, rho=rho, T=temperature,
                seed=seed)


def slab(box=(30.0, 30.0, 120.0), thickness=30.0, rho_l=0.73, rho_v=0.02, temperature=0.85,
         seed=3000, jitter=0.05, min_dist=0.8):
    """Vapour-liquid slab: an fcc liquid slab of the given thickness centred in z
    at density rho_l, vapour at rho_v inserted at random with a minimum spacing."""
    rng = np.random.default_rng(seed)
    box = np.asarray(box, dtype=np.float64)
    z0 = 0.5 * (box[2] - thickness)
    # liquid: fcc lattice of spacing set by rho_l, clipped to the slab
    a = (4.0 / rho_l) ** (1.0 / 3.0)
    mx = int(round(box[0] / a))
    my = int(round(box[1] / a))
    mz = int(round(thickness / a))
    ax, ay, az = box[0] / mx, box[1] / my, thickness / mz
    base = np.array([[0.0, 0.0, 0.0], [0.5, 0.5, 0.0], [0.5, 0.0, 0.5], [0.0, 0.5, 0.5]])
    gx, gy, gz = np.meshgrid(np.arange(mx), np.arange(my), np.arange(mz), indexing="ij")
    cells = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1).astype(np.float64)
    liq = (cells[:, None, :] + base[None]).reshape(-1, 3) * np.array([ax, ay, az])
    liq[:, 2] += z0
    liq += rng.uniform(-jitter, jitter, size=liq.shape)
    # vapour: random sequential insertion outside the slab
    vol_v = box[0] * box[1] * (box[2] - thickness)
    n_v = int(round(rho_v * vol_v))
    vap = np.zeros((0, 3))
    half = n_v // 2
    for k, (zlo, zhi) in enumerate([(0.0, z0 - 1.0), (z0 + thickness + 1.0, box[2])]):
        cnt = half if k == 0 else n_v - half
        vap = random_sequential(cnt, [0.0, 0.0, zlo], [box[0], box[1], zhi], min_dist, rng,
                                existing=vap, box=box)
    pts = np.mod(np.vstack([liq, vap]), box)
    n = pts.shape[0]
    v = maxwell_boltzmann(n, temperature, rng)
    return dict(x=np.ascontiguousarray(pts.T), v=v, box=box, n=n, T=temperature, seed=seed,
                n_liquid=liq.shape[0], n_vapour=vap.shape[0])


def replicas(count=64, n_lo=500, n_hi=20000, rho_lo=0.1, rho_hi=0.85, t_lo=0.7, t_hi=1.3,
             config_index=4):
    """Batch of independent replicas: N log-uniform in [n_lo, n_hi], rho and T
    uniform; every replica starts on an fcc lattice scaled to its cubic box
    (jitter +-0.05) with Maxwell-Boltzmann velocities."""
    out = []
    for r in range(count):
        rng = np.random.default_rng(config_index * 1000 + r)
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        rho = rng.uniform(rho_lo, rho_hi)
        temp = rng.uniform(t_lo, t_hi)
        box = (n / rho) ** (1.0 / 3.0)
        x = fcc_positions(n, box, rng, jitter=0.05)
        v = maxwell_boltzmann(n, temp, rng)
        out.append(dict(x=x, v=v, box=np.array([box, box, box]), n=n, rho=rho, T=temp,
                        seed=config_index * 1000 + r))
    return out


# The five workload recipes (reduced LJ units, nu = 0.073, r_c = 2.5).
CONFIGS = {
    "liquid_n1000": dict(n=1000, rho=0.8, T=1.0, seed=1000),
    "liquid_n32k": dict(n=32000, rho=0.8, T=1.0, seed=2000),
    "liquid_n256k": dict(n=256000, rho=0.8, T=1.0, seed=5000),
}


def config(name):
    c = CONFIGS[name]
    return homogeneous(c["n"], c["rho"], c["T"], c["seed"])


# ------------------------------------------------- surrogate test inputs

SUR_NDESC, SUR_NVEC, SUR_NOUT, SUR_NPARAM = 32, 48, 16, 7312


def sur_params(seed, wscale=0.3):
    """Random surrogate parameters (float32, the model's flat layout)."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, wscale, SUR_NPARAM).astype(np.float32)


def sur_rows(n, seed, mean=None, scale=None, tscale=0.1):
    """Random descriptor rows around (mean, scale), vectors and targets
    (float32), standing in for a data set in tests of the MLP alone."""
    rng = np.random.default_rng(seed)
    mean = np.zeros(SUR_NDESC) if mean is None else np.asarray(mean, dtype=np.float64)
    scale = np.ones(SUR_NDESC) if scale is None else np.asarray(scale, dtype=np.float64)
    D = (rng.normal(size=(n, SUR_NDESC)) * scale + mean).astype(np.float32)
    V = rng.normal(size=(n, SUR_NVEC)).astype(np.float32)
    T = (rng.normal(size=(n, 3)) * tscale).astype(np.float32)
    return D, V, T
