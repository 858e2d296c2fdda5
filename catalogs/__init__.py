"""Seeded synthetic point catalogues shaped like the paper's workloads.

This module is the one piece of code shared by the CPU oracle tests and the
CUDA path. It only draws random numbers and places points; it holds none of
the N-point method's arithmetic (no lattice quantisation, no distances, no
binning, no counting). Every generator takes an explicit integer seed and
uses NumPy's PCG64, so the same call returns the same catalogue on any host.

Positions are float64 in h^-1 Mpc inside [0, L) per axis; weights are
float32. Lattice coordinates are produced elsewhere, by each side's own
quantiser (lattice spacing 1/1024 h^-1 Mpc).

Workload recipes (the paper's own catalogues are not available, so these
stand in for them):

* ``uniform``: a Poisson (binomial) catalogue, the paper's random catalogues.
* ``neyman_scott``: clustered catalogue. Parents are uniform, each parent
  receives Poisson(mean_children) children displaced by an isotropic
  Gaussian of width ``sigma`` per axis. Parents are drawn until exactly
  ``n`` points exist; the last cluster is truncated. Periodic boxes wrap the
  children; open boxes discard children outside the box and keep drawing.
* ``lognormal``: lognormal density field (Gaussian field with power-law
  spectrum P(k) ~ k^slope, Gaussian smoothing, unit variance, exponentiated),
  sampled multinomially over grid cells with uniform placement in the cell.
* ``lattice_tetrahedra``: isolated copies of one integer tetrahedron, each
  copy either the shape itself or its mirror image, randomly rotated by a
  proper lattice rotation and placed on a coarse grid so that no two copies
  interact within ``min_spacing``.
"""
from __future__ import annotations

import itertools

import numpy as np

LATTICE_PER_MPC = 1024


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def uniform(n: int, box: float, seed: int) -> np.ndarray:
    """``n`` independent uniform points in [0, box)^3 (float64, shape (n, 3))."""
    rng = _rng(seed)
    return rng.uniform(0.0, box, size=(int(n), 3))


def neyman_scott(n: int, box: float, seed: int, mean_children: float = 10.0,
                 sigma: float = 2.0, periodic: bool = True) -> np.ndarray:
    """Neyman-Scott (Thomas) process with exactly ``n`` points."""
    rng = _rng(seed)
    n = int(n)
    out = np.empty((n, 3), dtype=np.float64)
    filled = 0
    batch = max(64, int(1.2 * n / mean_children) + 16)
    while filled < n:
        parents = rng.uniform(0.0, box, size=(batch, 3))
        counts = rng.poisson(mean_children, size=batch)
        kids = np.repeat(parents, counts, axis=0)
        kids += rng.normal(0.0, sigma, size=kids.shape)
        if periodic:
            kids = np.mod(kids, box)
            # np.mod can return exactly `box` for tiny negative inputs
            kids[kids >= box] = 0.0
        else:
            inside = np.all((kids >= 0.0) & (kids < box), axis=1)
            kids = kids[inside]
        take = min(n - filled, kids.shape[0])
        out[filled:filled + take] = kids[:take]
        filled += take
    return out


def lognormal(n: int, box: float, seed: int, grid: int = 256,
              slope: float = -1.5, smoothing: float = 2.0) -> np.ndarray:
    """Lognormal catalogue of exactly ``n`` points in a periodic box."""
    rng = _rng(seed)
    g = int(grid)
    white = rng.standard_normal((g, g, g))
    fk = np.fft.rfftn(white)
    kf = 2.0 * np.pi * np.fft.fftfreq(g, d=box / g)
    kz = 2.0 * np.pi * np.fft.rfftfreq(g, d=box / g)
    k2 = (kf[:, None, None] ** 2 + kf[None, :, None] ** 2 + kz[None, None, :] ** 2)
    with np.errstate(divide="ignore"):
        amp = np.where(k2 > 0, k2 ** (0.25 * slope), 0.0)
    amp *= np.exp(-0.5 * k2 * smoothing ** 2)
    field = np.fft.irfftn(fk * amp, s=(g, g, g))
    field -= field.mean()
    field /= field.std()
    dens = np.exp(field - 0.5).ravel()
    dens /= dens.sum()
    cells = rng.choice(dens.size, size=int(n), p=dens)
    iz = cells % g
    iy = (cells // g) % g
    ix = cells // (g * g)
    h = box / g
    pos = np.stack([ix, iy, iz], axis=1).astype(np.float64)
    pos += rng.uniform(0.0, 1.0, size=pos.shape)
    pos *= h
    pos[pos >= box] = 0.0
    return pos


def uniform_weights(n: int, seed: int, lo: float = 0.5, hi: float = 1.5) -> np.ndarray:
    """FP32 weights drawn from U(lo, hi)."""
    rng = _rng(seed)
    return rng.uniform(lo, hi, size=int(n)).astype(np.float32)


def _proper_rotations() -> list[np.ndarray]:
    """The 24 signed permutation matrices with determinant +1."""
    mats = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            m = np.zeros((3, 3), dtype=np.int64)
            for r, (c, s) in enumerate(zip(perm, signs)):
                m[r, c] = s
            if round(np.linalg.det(m)) == 1:
                mats.append(m)
    return mats


def lattice_tetrahedra(shape_u: np.ndarray, n_struct: int, mirrored_fraction: float,
                       box_u: int, min_spacing_u: int, seed: int):
    """Isolated integer tetrahedra on a lattice grid.

    ``shape_u`` is a (4, 3) integer array (lattice units). Each copy is the
    shape or its mirror (x -> -x), chosen so that exactly
    ``round(mirrored_fraction * n_struct)`` copies are mirrored; each copy is
    then rotated by a random proper lattice rotation, its vertices are listed
    in a random order, and it is translated to its own grid site. Grid sites
    are ``min_spacing_u`` apart plus the shape's extent, so vertices of
    different copies are always farther apart than ``min_spacing_u``.

    Returns (positions in h^-1 Mpc as float64 exactly equal to lattice/1024,
    lattice int64 coordinates, per-copy mirrored flags).
    """
    rng = _rng(seed)
    shape_u = np.asarray(shape_u, dtype=np.int64)
    rots = _proper_rotations()
    ext = int(np.abs(shape_u - shape_u[0]).max()) * 2 + 2
    step = int(min_spacing_u) + ext + 1
    per_side = int(box_u // step)
    if per_side ** 3 < n_struct:
        raise ValueError("box too small for the requested number of copies")
    n_mirror = int(round(mirrored_fraction * n_struct))
    flags = np.zeros(n_struct, dtype=bool)
    flags[rng.permutation(n_struct)[:n_mirror]] = True
    sites = rng.permutation(per_side ** 3)[:n_struct]
    pts = []
    for k in range(n_struct):
        v = shape_u - shape_u[0]
        if flags[k]:
            v = v * np.array([-1, 1, 1], dtype=np.int64)
        v = v @ rots[int(rng.integers(len(rots)))].T
        v = v[rng.permutation(4)]
        s = int(sites[k])
        origin = np.array([s // (per_side * per_side), (s // per_side) % per_side,
                           s % per_side], dtype=np.int64) * step + ext // 2 + 1
        pts.append(np.mod(v + origin, box_u))
    lat = np.concatenate(pts, axis=0)
    order = rng.permutation(lat.shape[0])
    lat = lat[order]
    return lat.astype(np.float64) / LATTICE_PER_MPC, lat, flags


# Named workloads. Each entry gives everything needed to draw the catalogue
# and the binning; counting is done by the caller.
WORKLOADS = {
    # 20k uniform points, periodic L=200, rmax 20 in 10 bins: small parity case
    "uniform20k_L200_r20_nb10": dict(kind="uniform", n=20_000, box=200.0, periodic=True,
                                     rmin=0.0, rmax=20.0, nb=10, seed=0),
    # 1e6 Neyman-Scott data + 3e6 uniform randoms, periodic L=1000, rmax 40 in 20 bins
    "ns1M_L1000_r40_nb20": dict(kind="neyman_scott", n=1_000_000, box=1000.0, periodic=True,
                                rmin=0.0, rmax=40.0, nb=20, seed=1, sigma=2.0,
                                randoms=3_000_000, random_seed=2, weight_seed=3),
    # 2e5 Neyman-Scott points, periodic L=400, rmax 30 in 8 bins (4pCF + parity)
    "ns200k_L400_r30_nb8": dict(kind="neyman_scott", n=200_000, box=400.0, periodic=True,
                                rmin=0.0, rmax=30.0, nb=8, seed=4, sigma=2.0),
    # 1e5 Neyman-Scott data + 1e5 uniform randoms (1:1), periodic L=400, rmax 30 in 8
    # bins: the connected 4pCF with signed weights
    "ns100k_r100k_L400_r30_nb8": dict(kind="neyman_scott", n=100_000, box=400.0, periodic=True,
                                      rmin=0.0, rmax=30.0, nb=8, seed=6, sigma=2.0,
                                      randoms=100_000, random_seed=7, weight_seed=8),
    # 1e6 Neyman-Scott (sigma 5), open box L=1494, rmax 150 in 15 bins (out-of-core)
    "ns1M_open_L1494_r150_nb15": dict(kind="neyman_scott", n=1_000_000, box=1494.0,
                                      periodic=False, rmin=0.0, rmax=150.0, nb=15, seed=5,
                                      sigma=5.0),
}


def bin_edges_u(rmin: float, rmax: float, nb: int) -> np.ndarray:
    """Integer bin edges in lattice units, rounding half up in exact rationals.

    E_b = floor(1024 * (rmin + b * (rmax - rmin) / nb) + 1/2), evaluated with
    Python integers/fractions so the edges do not depend on float rounding.
    """
    from fractions import Fraction
    lo = Fraction(rmin).limit_denominator(1 << 20)
    hi = Fraction(rmax).limit_denominator(1 << 20)
    out = []
    for b in range(nb + 1):
        x = LATTICE_PER_MPC * (lo + b * (hi - lo) / nb) + Fraction(1, 2)
        out.append(x.numerator // x.denominator)
    return np.asarray(out, dtype=np.int64)


def draw(name: str, **overrides):
    """Draw a named workload; returns dict(pos, box, periodic, edges_u, ...)."""
    spec = dict(WORKLOADS[name])
    spec.update(overrides)
    kind = spec["kind"]
    if kind == "uniform":
        pos = uniform(spec["n"], spec["box"], spec["seed"])
    elif kind == "neyman_scott":
        pos = neyman_scott(spec["n"], spec["box"], spec["seed"], sigma=spec.get("sigma", 2.0),
                           periodic=spec["periodic"])
    elif kind == "lognormal":
        pos = lognormal(spec["n"], spec["box"], spec["seed"], grid=spec.get("grid", 256))
    else:
        raise ValueError(kind)
    spec["pos"] = pos
    spec["edges_u"] = bin_edges_u(spec["rmin"], spec["rmax"], spec["nb"])
    spec["box_u"] = int(round(spec["box"] * LATTICE_PER_MPC))
    return spec
