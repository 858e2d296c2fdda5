"""Pins of the oracle's configuration tooling: the Cayley-Menger mask
(Sec. 5.2) and exact fine-to-coarse rebinning (Sec. 5.1)."""
import json
import os

import numpy as np
import pytest

import catalogs
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_cm_mask_reproduces_printed_count():
    """4 radial bins over 20-65 h^-1Mpc: 178 of 276 orbits are realisable."""
    gold = json.load(open(os.path.join(GOLDEN, "config_counts.json")))["cayley_menger"]
    nb = gold["nb"]
    edges = [int(20 * 1024 + b * 11.25 * 1024) for b in range(nb + 1)]
    centres = [(edges[b] + edges[b + 1]) / 2048 for b in range(nb)]
    assert centres == gold["centres_mpc"]
    mask = oracle.config_mask_cm(nb, edges)
    assert len(mask) == 276
    assert int(mask.sum()) == gold["realisable"]


def test_cm_determinant_closed_forms():
    # regular tetrahedron of side a: 288 V^2 = 288 (a^3 / (6 sqrt 2))^2 = 4 a^6
    for a in (1, 3, 26):
        assert oracle.cayley_menger_det([a * a] * 6) == 4 * a ** 6
    # right corner with legs p, q, r at vertex 0: V = pqr / 6, 288 V^2 = 8 p^2 q^2 r^2
    p, q, r = 3, 5, 7
    d2 = [p * p, q * q, r * r, p * p + q * q, p * p + r * r, q * q + r * r]
    assert oracle.cayley_menger_det(d2) == 8 * p * p * q * q * r * r
    # four coplanar points (unit square): zero volume
    assert oracle.cayley_menger_det([1, 2, 1, 1, 2, 1]) == 0
    # five edges a and one x: flat when x^2 = 3 a^2 (two equilateral faces
    # folded open), realisable below, not above; the printed example of five
    # 26 h^-1Mpc edges and one of 48 falls above
    a = 26
    assert oracle.cayley_menger_det([a * a] * 5 + [3 * a * a]) == 0
    assert oracle.cayley_menger_det([a * a] * 5 + [3 * a * a - 1]) > 0
    assert oracle.cayley_menger_det([a * a] * 5 + [3 * a * a + 1]) < 0
    assert oracle.cayley_menger_det([a * a] * 5 + [48 * 48]) < 0
    # a face violating the triangle inequality is not realisable
    assert oracle.cayley_menger_det([1, 1, 1, 9, 1, 1]) <= 0


def test_cm_mask_label_invariant():
    """The mask depends on the orbit, not on which representative is used."""
    nb = 3
    edges = [0, 5000, 9000, 12000]
    mask = oracle.config_mask_cm(nb, edges)
    centre2 = [((edges[b] + edges[b + 1]) / 2) ** 2 for b in range(nb)]
    import itertools
    for o in range(len(mask)):
        rep, _ = oracle.config_bins(4, nb, o)
        for perm in itertools.permutations(range(4)):
            t = oracle._relabel(rep, perm)
            assert (oracle.cayley_menger_det([centre2[b] for b in t]) > 0) == bool(mask[o])


@pytest.fixture(scope="module")
def clustered():
    L = 80.0
    box_u = int(L * 1024)
    X = oracle.quantize(catalogs.neyman_scott(5000, L, seed=301, sigma=1.5), box_u, True)
    w = catalogs.uniform_weights(len(X), seed=302)
    return X, box_u, w


def test_rebin_3pcf_equals_direct_coarse_count(clustered):
    """Fine bins 0.75 h^-1Mpc wide over 0-9; coarse bins 1.5 wide over
    1.5-7.5. Rebinning the fine counts must give exactly the counts taken
    directly on the coarse edges: both select the same triangles."""
    X, box_u, w = clustered
    fine = np.array([int(768 * k) for k in range(13)], dtype=np.int64)
    coarse = fine[2:11:2]
    bin_map = np.full(12, -1, dtype=np.int32)
    for k in range(2, 10):
        bin_map[k] = (k - 2) // 2
    fc, fw = oracle.Graph(X, box_u, fine).count_3pcf(w)
    cc, cw = oracle.Graph(X, box_u, coarse).count_3pcf(w)
    rc, rw = oracle.rebin_3pcf(12, 4, bin_map, fc, fw)
    assert cc.sum() > 10_000
    assert np.array_equal(rc, cc)
    np.testing.assert_allclose(rw, cw, rtol=1e-12)


def test_rebin_4pcf_equals_direct_coarse_count(clustered):
    """As above for the parity 4pCF: even, odd and weighted channels, with
    fine bins dropped at both ends."""
    X, box_u, w = clustered
    fine = np.array([0, 1200, 2300, 3500, 4600, 5800, 7000], dtype=np.int64)
    coarse = np.array([1200, 3500, 5800], dtype=np.int64)
    bin_map = np.array([-1, 0, 0, 1, 1, -1], dtype=np.int32)
    fe, fo, fwe, fwo = oracle.Graph(X, box_u, fine).count_4pcf(w)
    ce, co, cwe, cwo = oracle.Graph(X, box_u, coarse).count_4pcf(w)
    re, ro, rwe, rwo = oracle.rebin_4pcf(6, 2, bin_map, fe, fo, fwe, fwo)
    assert ce.sum() > 10_000 and np.abs(co).sum() > 0
    assert np.array_equal(re, ce)
    assert np.array_equal(ro, co)
    np.testing.assert_allclose(rwe, cwe, rtol=1e-12)
    np.testing.assert_allclose(rwo, cwo, rtol=1e-12, atol=1e-12 * np.abs(cwe).max())


def test_rebin_identity_map():
    nb = 3
    rng = np.random.default_rng(5)
    n4 = oracle.num_configs(4, nb)
    e = rng.integers(0, 1000, n4).astype(np.uint64)
    o = rng.integers(-50, 50, n4)
    chiral = np.array([oracle.config_bins(4, nb, c)[1] for c in range(n4)])
    o[~chiral] = 0
    re, ro, _, _ = oracle.rebin_4pcf(nb, nb, np.arange(nb), e, o)
    assert np.array_equal(re, e) and np.array_equal(ro, o)
    n3 = oracle.num_configs(3, nb)
    c3 = rng.integers(0, 1000, n3).astype(np.uint64)
    assert np.array_equal(oracle.rebin_3pcf(nb, nb, np.arange(nb), c3), c3)


def test_equilateral_brute_force():
    """All triples of a tiny catalogue: triangles whose three pair bins agree."""
    import itertools

    from tests import bruteforce
    rng = np.random.default_rng(17)
    box_u = 20_000
    X = rng.integers(0, box_u, size=(90, 3)).astype(np.int32)
    w = catalogs.uniform_weights(len(X), seed=18)
    edges = np.array([0, 2000, 3500, 5000], dtype=np.int64)
    B = bruteforce.bin_matrix(X, box_u, edges)
    want = np.zeros(3, np.uint64)
    wsum = np.zeros(3)
    for i, j, k in itertools.combinations(range(len(X)), 3):
        if B[i, j] >= 0 and B[i, j] == B[i, k] == B[j, k]:
            want[B[i, j]] += 1
            wsum[B[i, j]] += float(w[i]) * float(w[j]) * float(w[k])
    c, ws = oracle.equilateral_3pcf(oracle.Graph(X, box_u, edges), w)
    assert want.sum() > 20
    assert np.array_equal(c, want)
    np.testing.assert_allclose(ws, wsum, rtol=1e-12)
