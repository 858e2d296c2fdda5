"""Pins of the oracle's anisotropic (mu-binned) 3pCF.

The paper names mu binning for redshift-space distortions without defining
it; the reading pinned here: line of sight along z, a triangle's mu is
|n_z| / |n| for the normal n of its plane, bin floor(nmu mu) (mu = 1 in the
last bin), collinear triangles in the extra bin nmu. The pins: the
all-triples brute force (normal taken from another vertex, bin from integer
square roots), hand-built triangles whose mu is known exactly (including a
mu that lies on a bin edge), the plain 3pCF as the sum over mu bins, a
rotation about the line of sight that must change nothing, a planted
anisotropic structure that a swap of axes must move, and the flat mu
distribution of isotropic triangles.
"""
import numpy as np
import pytest

import catalogs
import oracle
from tests import bruteforce as bf


def rand_lattice(n, box_u, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, box_u, size=(n, 3)).astype(np.int32)


def conf_index(nb, bins):
    return bf.configs3(nb)[tuple(sorted(bins))]


@pytest.mark.parametrize("periodic,nmu,seed", [(True, 4, 1), (False, 5, 2), (True, 7, 3)])
def test_mu_counts_match_brute_force(periodic, nmu, seed):
    box_u = 40_000
    X = np.concatenate([rand_lattice(110, box_u, seed),
                        # a clump, so that small triangles and repeated
                        # directions occur
                        np.mod(20_000 + np.random.default_rng(seed + 9).integers(
                            -2500, 2501, size=(40, 3)), box_u).astype(np.int32)])
    edges = np.array([0, 3000, 6000, 9000], dtype=np.int64)
    bu = box_u if periodic else 0
    w = catalogs.uniform_weights(len(X), seed=seed + 20)
    w[::3] *= -1.0
    og = oracle.Graph(X, bu, edges)
    c, s = og.count_3pcf_mu(nmu, w)
    bc, bs = bf.count3_mu(X, bu, edges, nmu, w)
    assert c.sum() > 50
    assert np.array_equal(c, bc)
    assert np.array_equal(s, bs)
    assert np.array_equal(og.count_3pcf_mu(nmu), bc)


def test_mu_of_hand_built_triangles():
    box_u = 100_000
    edges = np.array([0, 2000, 4000, 6000], dtype=np.int64)
    P = np.array([50_000, 50_000, 50_000])

    def one(j, k, nmu):
        X = np.array([P, P + j, P + k], dtype=np.int32)
        return oracle.Graph(X, box_u, edges).count_3pcf_mu(nmu)

    # in the xy plane: normal along z, mu = 1, the last bin
    c = one([3000, 0, 0], [0, 3000, 0], 4)
    assert c.sum() == 1 and c[conf_index(3, (1, 1, 2)), 3] == 1
    # in the xz plane: normal along y, mu = 0
    c = one([3000, 0, 0], [0, 0, 3000], 4)
    assert c[conf_index(3, (1, 1, 2)), 0] == 1
    # collinear: the extra bin
    c = one([2500, 0, 0], [5000, 0, 0], 4)
    assert c.sum() == 1 and c[conf_index(3, (1, 1, 2)), 4] == 1
    # normal along (4, 0, 3): mu = 3/5 exactly, on the edge between bins 2
    # and 3 of five; the edge belongs to the bin above it
    c = one([0, 3000, 0], [1800, 0, -2400], 5)
    assert c.sum() == 1 and c[conf_index(3, (1, 1, 2)), 3] == 1
    # the same triangle with nmu = 10: mu = 0.6 = 6/10, bin 6
    c = one([0, 3000, 0], [1800, 0, -2400], 10)
    assert c[conf_index(3, (1, 1, 2)), 6] == 1
    # a normal just below 3/5 (4, 0, 3) -> (4001, 0, 3000): bin 2 of five
    u, v = np.array([0, 3000, 0]), np.array([3000, 0, -4001])
    assert np.cross(u, v).tolist() == [-12003000, 0, -9000000]
    c = one(u.tolist(), v.tolist(), 5)
    assert c[conf_index(3, (1, 2, 2)), 2] == 1


def test_mu_bins_sum_to_the_3pcf():
    box_u = 120_000
    X = np.concatenate([rand_lattice(6000, box_u, 11),
                        np.mod(60_000 + np.random.default_rng(12).integers(
                            -6000, 6001, size=(1500, 3)), box_u).astype(np.int32)])
    edges = np.array([0, 2000, 4000, 6000, 8000], dtype=np.int64)
    og = oracle.Graph(X, box_u, edges)
    w = catalogs.uniform_weights(len(X), seed=13)
    c, s = og.count_3pcf_mu(6, w)
    c3, s3 = og.count_3pcf(w)
    assert np.array_equal(c.sum(axis=1), c3)
    np.testing.assert_allclose(s.sum(axis=1), s3, rtol=1e-12)


def test_rotation_about_the_line_of_sight_changes_nothing():
    box_u = 90_000
    X = rand_lattice(5000, box_u, 21)
    edges = np.array([1000, 3000, 5000, 7000], dtype=np.int64)
    # (x, y, z) -> (L - 1 - y, x, z): a quarter turn about z, a lattice map
    R = np.stack([box_u - 1 - X[:, 1], X[:, 0], X[:, 2]], axis=1).astype(np.int32)
    a = oracle.Graph(X, box_u, edges).count_3pcf_mu(8)
    b = oracle.Graph(R, box_u, edges).count_3pcf_mu(8)
    assert np.array_equal(a, b)
    # z -> -z (mirror through the xy plane) changes nothing either
    M = np.stack([X[:, 0], X[:, 1], box_u - 1 - X[:, 2]], axis=1).astype(np.int32)
    assert np.array_equal(oracle.Graph(M, box_u, edges).count_3pcf_mu(8), a)


def test_planted_planar_structure_moves_with_the_axes():
    """Flat triangles in planes z = const sit in the top mu bin; swapping x
    and z moves them to the bottom bin."""
    box_u = 200_000
    rng = np.random.default_rng(31)
    pts = []
    # cluster centres 40,000 apart: no edge joins two clusters
    grid = 20_000 + 40_000 * np.stack(np.meshgrid(*[np.arange(4)] * 3), axis=-1).reshape(-1, 3)
    for c in grid:
        for _ in range(5):
            pts.append([c[0] + rng.integers(-1500, 1501), c[1] + rng.integers(-1500, 1501), c[2]])
    X = np.array(pts, dtype=np.int32)
    edges = np.array([200, 1500, 3000, 4500], dtype=np.int64)
    nmu = 4
    a = oracle.Graph(X, box_u, edges).count_3pcf_mu(nmu).sum(axis=0)
    S = X[:, [2, 1, 0]].copy()
    b = oracle.Graph(S, box_u, edges).count_3pcf_mu(nmu).sum(axis=0)
    assert a.sum() > 500 and a.sum() == b.sum()
    assert a[nmu - 1] + a[nmu] == a.sum()  # mu = 1 or collinear
    assert b[0] + b[nmu] == b.sum()
    assert a[nmu] == b[nmu]


def test_isotropic_triangles_have_flat_mu():
    """For isotropic orientations mu = |cos| of the normal's polar angle is
    uniform on [0, 1]: the bins hold equal shares within Poisson noise."""
    box_u = 160_000
    X = rand_lattice(30_000, box_u, 41)
    edges = np.array([2000, 4000, 6000, 8000], dtype=np.int64)
    nmu = 5
    c = oracle.Graph(X, box_u, edges).count_3pcf_mu(nmu).sum(axis=0)
    tot = c[:nmu].sum()
    assert tot > 200_000
    # triangles of one catalogue share vertices, so allow a generous band
    sigma = np.sqrt(tot / nmu)
    assert np.all(np.abs(c[:nmu] - tot / nmu) < 6 * sigma)
    assert c[nmu] < 1e-3 * tot
