"""Brute-force reference for tiny inputs, used to pin the oracle.

Everything here is written from the definitions with Python integers and
itertools, independently of ``oracle/`` and of the CUDA library: all pairs
for the graph, all triples for triangles, networkx clique enumeration for
tetrahedra, all 24 vertex relabellings for the 4-point configuration, and
exact Python-integer determinants for the parity volume.
"""
from __future__ import annotations

import functools
import itertools
import math
from fractions import Fraction

import numpy as np


def displacements(X: np.ndarray, box_u: int) -> np.ndarray:
    """(N, N, 3) int64 minimum-image displacements X_j - X_i."""
    X = X.astype(np.int64)
    d = X[None, :, :] - X[:, None, :]
    if box_u > 0:
        d = np.where(2 * d >= box_u, d - box_u, d)
        d = np.where(2 * d < -box_u, d + box_u, d)
    return d


def bin_matrix(X: np.ndarray, box_u: int, edges_u) -> np.ndarray:
    """(N, N) int matrix: bin of the pair, or -1 when the pair is not an edge."""
    d = displacements(X, box_u)
    D2 = (d * d).sum(axis=2)
    e2 = np.asarray(edges_u, dtype=np.int64) ** 2
    nb = len(e2) - 1
    B = np.full(D2.shape, -1, dtype=np.int64)
    for b in range(nb):
        B[(D2 >= e2[b]) & (D2 < e2[b + 1])] = b
    np.fill_diagonal(B, -1)
    return B


def configs3(nb: int):
    reps = [t for t in itertools.product(range(nb), repeat=3) if t[0] <= t[1] <= t[2]]
    return {t: k for k, t in enumerate(sorted(reps))}


SLOTS = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
PERMS = list(itertools.permutations(range(4)))


def perm_sign(p) -> int:
    inv = sum(1 for a in range(4) for b in range(a + 1, 4) if p[a] > p[b])
    return -1 if inv % 2 else 1


def canonical4(bins_of_pair):
    """Smallest relabelled tuple and one relabelling reaching it.

    ``bins_of_pair(a, b)`` gives the bin of the edge between vertices a, b of
    the input labelling; relabelling p puts old vertex p[k] at new label k.
    """
    best, bestp = None, None
    for p in PERMS:
        t = tuple(bins_of_pair(p[a], p[b]) for a, b in SLOTS)
        if best is None or t < best:
            best, bestp = t, p
    return best, bestp


def configs4(nb: int):
    """Orbit representatives in lexicographic order -> (rank, chiral)."""
    reps = set()
    for t in itertools.product(range(nb), repeat=6):
        def f(a, b, t=t):
            a, b = min(a, b), max(a, b)
            return t[SLOTS.index((a, b))]
        reps.add(canonical4(f)[0])
    out = {}
    for k, r in enumerate(sorted(reps)):
        def f(a, b, r=r):
            a, b = min(a, b), max(a, b)
            return r[SLOTS.index((a, b))]
        chiral = all(perm_sign(p) > 0 for p in PERMS
                     if tuple(f(p[a], p[b]) for a, b in SLOTS) == r)
        out[r] = (k, chiral)
    return out


def det3(u, v, w) -> int:
    return (u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0]) +
            u[2] * (v[0] * w[1] - v[1] * w[0]))


def count3(X, box_u, edges_u, w=None):
    nb = len(edges_u) - 1
    B = bin_matrix(X, box_u, edges_u)
    conf = configs3(nb)
    counts = np.zeros(len(conf), dtype=np.uint64)
    wsum = [Fraction(0)] * len(conf)
    n = X.shape[0]
    for i, j, k in itertools.combinations(range(n), 3):
        if B[i, j] < 0 or B[i, k] < 0 or B[j, k] < 0:
            continue
        c = conf[tuple(sorted((int(B[i, j]), int(B[i, k]), int(B[j, k]))))]
        counts[c] += 1
        if w is not None:
            wsum[c] += Fraction(float(w[i])) * Fraction(float(w[j])) * Fraction(float(w[k]))
    if w is None:
        return counts
    return counts, np.array([float(x) for x in wsum])


def count4(X, box_u, edges_u, w=None):
    """Even/odd 4-point counts via networkx 4-cliques."""
    import networkx as nx
    nb = len(edges_u) - 1
    B = bin_matrix(X, box_u, edges_u)
    d = displacements(X, box_u)
    conf = configs4(nb)
    G = nx.Graph()
    G.add_nodes_from(range(X.shape[0]))
    ii, jj = np.nonzero(np.triu(B >= 0, 1))
    G.add_edges_from(zip(ii.tolist(), jj.tolist()))
    even = np.zeros(len(conf), dtype=np.uint64)
    odd = np.zeros(len(conf), dtype=np.int64)
    weven = [Fraction(0)] * len(conf)
    wodd = [Fraction(0)] * len(conf)
    for cl in nx.enumerate_all_cliques(G):
        if len(cl) < 4:
            continue
        if len(cl) > 4:
            break
        v = list(cl)
        rep, p = canonical4(lambda a, b: int(B[v[a], v[b]]))
        k, chiral = conf[rep]
        even[k] += 1
        wt = Fraction(1)
        if w is not None:
            for x in v:
                wt *= Fraction(float(w[x]))
            weven[k] += wt
        if chiral:
            u = [v[p[t]] for t in range(4)]
            vecs = [[int(d[u[0], u[t], a]) for a in range(3)] for t in (1, 2, 3)]
            V = det3(*vecs)
            if V != 0:
                s = 1 if V > 0 else -1
                odd[k] += s
                wodd[k] += s * wt
    if w is None:
        return even, odd
    return even, odd, np.array([float(x) for x in weven]), np.array([float(x) for x in wodd])


def pairs(X, box_u, edges_u, w=None):
    nb = len(edges_u) - 1
    B = bin_matrix(X, box_u, edges_u)
    out = np.zeros(nb, dtype=np.uint64)
    wout = [Fraction(0)] * nb
    n = X.shape[0]
    for i in range(n):
        for j in range(i + 1, n):
            if B[i, j] >= 0:
                out[B[i, j]] += 1
                if w is not None:
                    wout[B[i, j]] += Fraction(float(w[i])) * Fraction(float(w[j]))
    if w is None:
        return out
    return out, np.array([float(x) for x in wout])


def rows(X, box_u, edges_u):
    """Sorted neighbour rows as a list of (ids, bins)."""
    B = bin_matrix(X, box_u, edges_u)
    out = []
    for i in range(X.shape[0]):
        j = np.nonzero(B[i] >= 0)[0]
        out.append((j.astype(np.int64), B[i, j].astype(np.int64)))
    return out


# ----------------------------------------------------------------------------
# Pixelised directions (the reading of Sec. 3.2 used here: 256 equal-area
# pixels, 16 bands of equal width in cos(theta) times 16 sectors of equal
# width in phi), restated independently with high-precision arithmetic.


@functools.lru_cache(maxsize=None)
def direction_pixel(x: int, y: int, z: int) -> int:
    """Band from cos(theta) = z/|d| (16 bands of width 1/8 on [-1, 1], a
    value on a band edge belongs to the upper band), sector from
    phi = atan2(y, x) in [0, 2 pi) (16 sectors of pi/8, an edge belongs to
    the upper sector); sector 0 on the z axis. Computed with mpmath at 60
    digits; the only directions exactly on an edge are z = 0 (band edge) and
    the axes and diagonals of the x-y plane (sector edges), handled exactly."""
    import mpmath
    mpmath.mp.dps = 60
    x, y, z = int(x), int(y), int(z)
    if z == 0:
        band = 8
    else:
        c = mpmath.mpf(z) / mpmath.sqrt(mpmath.mpf(x * x + y * y + z * z))
        band = min(15, int(mpmath.floor((c + 1) * 8)))
    if x == 0 and y == 0:
        sector = 0
    elif x == 0 or y == 0 or abs(x) == abs(y):
        # exactly on a multiple of pi/4
        eighth = {(1, 0): 0, (1, 1): 1, (0, 1): 2, (-1, 1): 3, (-1, 0): 4, (-1, -1): 5,
                  (0, -1): 6, (1, -1): 7}
        sgn = lambda v: (v > 0) - (v < 0)  # noqa: E731
        sector = 2 * eighth[(sgn(x), sgn(y))]
    else:
        phi = mpmath.atan2(y, x)
        if phi < 0:
            phi += 2 * mpmath.pi
        sector = int(mpmath.floor(phi / (mpmath.pi / 8)))
    return 16 * band + sector


def pixel_centre(p: int):
    import math
    band, sector = divmod(p, 16)
    zc = -1.0 + (band + 0.5) / 8.0
    phi = (sector + 0.5) * math.pi / 8.0
    rho = math.sqrt(1.0 - zc * zc)
    return (rho * math.cos(phi), rho * math.sin(phi), zc)


def pixel_volume(p1: int, p2: int, p3: int) -> float:
    a, b, c = pixel_centre(p1), pixel_centre(p2), pixel_centre(p3)
    cx = a[1] * b[2] - a[2] * b[1]
    cy = a[2] * b[0] - a[0] * b[2]
    cz = a[0] * b[1] - a[1] * b[0]
    return cx * c[0] + cy * c[1] + cz * c[2]


def count4_pixel(X, box_u, edges_u):
    """Even/odd 4-point counts with the odd sign from pixelised directions:
    the tetrahedron's vertices in ascending index order (o, v1, v2, v3), the
    spokes o -> vk, V = pixel volume of their pixels; odd += sign(V) times
    the parity of a relabelling onto the orbit representative, when the orbit
    is chiral and |V| >= 1e-9."""
    import networkx as nx
    nb = len(edges_u) - 1
    B = bin_matrix(X, box_u, edges_u)
    d = displacements(X, box_u)
    conf = configs4(nb)
    G = nx.Graph()
    G.add_nodes_from(range(X.shape[0]))
    ii, jj = np.nonzero(np.triu(B >= 0, 1))
    G.add_edges_from(zip(ii.tolist(), jj.tolist()))
    even = np.zeros(len(conf), dtype=np.uint64)
    odd = np.zeros(len(conf), dtype=np.int64)
    for cl in nx.enumerate_all_cliques(G):
        if len(cl) < 4:
            continue
        if len(cl) > 4:
            break
        v = sorted(cl)
        rep, p = canonical4(lambda a, b: int(B[v[a], v[b]]))
        k, chiral = conf[rep]
        even[k] += 1
        if chiral:
            spokes = [tuple(int(t) for t in d[v[0], v[m]]) for m in (1, 2, 3)]
            if any(s == (0, 0, 0) for s in spokes):
                continue  # coincident points: no direction, degenerate
            V = pixel_volume(*(direction_pixel(*s) for s in spokes))
            if abs(V) >= 1e-9:
                odd[k] += (1 if V > 0 else -1) * perm_sign(p)
    return even, odd


def count3_mu(X, box_u, edges_u, nmu, w=None):
    """Anisotropic 3pCF by brute force: every triangle's mu is |n_z| / |n|
    for the normal of its plane, taken here from the middle vertex j
    (n = d(j, i) x d(j, k), the same line as from any vertex);
    bin = floor(nmu mu) (at most nmu - 1) via integer square roots;
    collinear triangles in bin nmu."""
    nb = len(edges_u) - 1
    B = bin_matrix(X, box_u, edges_u)
    d = displacements(X, box_u)
    conf = configs3(nb)
    counts = np.zeros((len(conf), nmu + 1), dtype=np.uint64)
    wsum = [[Fraction(0)] * (nmu + 1) for _ in conf]
    n = X.shape[0]
    for i, j, k in itertools.combinations(range(n), 3):
        if B[i, j] < 0 or B[i, k] < 0 or B[j, k] < 0:
            continue
        u = [int(x) for x in d[j, i]]
        v = [int(x) for x in d[j, k]]
        nv = (u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0])
        n2 = nv[0] ** 2 + nv[1] ** 2 + nv[2] ** 2
        if n2 == 0:
            m = nmu
        else:
            m = min(nmu - 1, math.isqrt((nmu * nmu * nv[2] * nv[2]) // n2))
        c = conf[tuple(sorted((int(B[i, j]), int(B[i, k]), int(B[j, k]))))]
        counts[c, m] += 1
        if w is not None:
            wsum[c][m] += Fraction(float(w[i])) * Fraction(float(w[j])) * Fraction(float(w[k]))
    if w is None:
        return counts
    return counts, np.array([[float(x) for x in row] for row in wsum])
