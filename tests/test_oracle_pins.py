"""Pins of the CPU oracle against things other than itself.

Each test ties an oracle function to the paper's printed numbers, to a
closed form, to an invariance of the definition, or to the brute-force
reference in ``bruteforce.py`` (all triples / networkx 4-cliques / all 24
relabellings, written independently of the oracle).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import catalogs
import oracle
from tests import bruteforce as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def load_golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def rand_lattice(n, box_u, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, box_u, size=(n, 3)).astype(np.int32)


def clustered_lattice(n, box_u, seed, spread):
    rng = np.random.default_rng(seed)
    centres = rng.integers(0, box_u, size=(max(1, n // 8), 3))
    pick = centres[rng.integers(0, centres.shape[0], size=n)]
    X = pick + rng.integers(-spread, spread + 1, size=(n, 3))
    return np.mod(X, box_u).astype(np.int32)


# --------------------------------------------------------------------------
# a1: quantisation


def test_quantize_hand_values():
    box_u = 1024 * 10
    pos = np.array([[0.0, 1.0 / 1024, 9.9999999],
                    [-1.0 / 1024, 10.0, 5.0004],
                    [3.25, 7.0, 0.5]])
    X = oracle.quantize(pos, box_u, periodic=True)
    assert X.tolist() == [[0, 1, 10239], [10239, 0, 5120], [3328, 7168, 512]]
    with pytest.raises(ValueError):
        oracle.quantize(np.array([[-1e-9, 0.0, 0.0]]), box_u, periodic=False)
    with pytest.raises(ValueError):
        oracle.quantize(np.array([[10.0, 0.0, 0.0]]), box_u, periodic=False)


# --------------------------------------------------------------------------
# a2: graph


def adversarial_points(box_u, edges_u):
    """Coincident points, points at exactly each bin edge, and half-box pairs."""
    pts = [[100, 100, 100], [100, 100, 100]]  # coincident: d = 0
    base = np.array([box_u // 3, box_u // 5, box_u // 7])
    for e in edges_u:
        pts.append((base + [int(e), 0, 0]).tolist())
        pts.append((base + [0, int(e) - 1, 0]).tolist())
    pts.append([0, 0, 0])
    pts.append([box_u // 2, 0, 0])  # exactly half a box apart
    pts.append([box_u - 1, box_u - 1, box_u - 1])  # wraps next to the origin
    return np.mod(np.array(pts, dtype=np.int64), box_u).astype(np.int32)


@pytest.mark.parametrize("periodic", [True, False])
def test_graph_matches_all_pairs(periodic):
    box_u = 40_000
    edges_u = np.array([0, 1500, 3000, 4500, 6000, 9000], dtype=np.int64)
    X = np.concatenate([rand_lattice(300, box_u, 1), clustered_lattice(200, box_u, 2, 2500),
                        adversarial_points(box_u, edges_u)])
    bu = box_u if periodic else 0
    ref = bf.rows(X, bu, edges_u)
    for method in ("brute", "grid"):
        g = oracle.Graph(X, bu, edges_u, method=method, nthreads=4)
        ptr, nbr, b = g.export()
        for i, (ids, bins) in enumerate(ref):
            assert np.array_equal(nbr[ptr[i]:ptr[i + 1]], ids), (method, i)
            assert np.array_equal(b[ptr[i]:ptr[i + 1]], bins), (method, i)


def test_graph_edge_semantics():
    """Half-open bins on squared integer distances, coincident points in bin 0."""
    box_u = 100_000
    edges_u = np.array([0, 1000, 2000], dtype=np.int64)
    X = np.array([[10, 10, 10], [10, 10, 10], [1010, 10, 10], [10, 2010, 10], [10, 10, 1009]],
                 dtype=np.int32)
    g = oracle.Graph(X, box_u, edges_u, method="brute", nthreads=1)
    ptr, nbr, b = g.export()
    row0 = dict(zip(nbr[ptr[0]:ptr[1]].tolist(), b[ptr[0]:ptr[1]].tolist()))
    # d=0 -> bin 0; d=1000 -> bin 1 (lower edge inclusive); d=2000 -> not an edge
    # (upper edge exclusive); d=999 -> bin 0
    assert row0 == {1: 0, 2: 1, 4: 0}


# --------------------------------------------------------------------------
# a3: triangles


@pytest.mark.parametrize("periodic,seed", [(True, 3), (False, 4), (True, 5)])
def test_3pcf_matches_all_triples(periodic, seed):
    box_u = 30_000
    edges_u = np.array([0, 2000, 3500, 5000, 7000], dtype=np.int64)
    X = np.concatenate([rand_lattice(90, box_u, seed), clustered_lattice(60, box_u, seed + 10, 3000)])
    bu = box_u if periodic else 0
    ref = bf.count3(X, bu, edges_u)
    assert ref.sum() > 50
    g = oracle.Graph(X, bu, edges_u, nthreads=3)
    assert np.array_equal(g.count_3pcf(), ref)


def test_3pcf_weighted_exact():
    box_u = 30_000
    edges_u = np.array([0, 2500, 5000, 7000], dtype=np.int64)
    X = clustered_lattice(100, box_u, 7, 4000)
    w = catalogs.uniform_weights(X.shape[0], seed=9)
    ref_c, ref_w = bf.count3(X, box_u, edges_u, w)
    g = oracle.Graph(X, box_u, edges_u, nthreads=2)
    c, ws = g.count_3pcf(w)
    assert np.array_equal(c, ref_c)
    # exact sums rounded once, to nearest: bit for bit the rational sums
    assert np.array_equal(ws, ref_w)
    # unit weights reproduce the counts; doubling every weight scales by 8
    c1, w1 = g.count_3pcf(np.ones(X.shape[0], np.float32))
    assert np.array_equal(w1, c1.astype(np.float64))
    _, w2 = g.count_3pcf(2 * w)
    assert np.array_equal(w2, 8 * ws)


def test_3pcf_signed_weights_exact():
    """Weights of both signs (the signed estimator's case): the oracle's exact
    sums against exact rational sums over all triples."""
    box_u = 30_000
    edges_u = np.array([0, 2500, 5000, 7000], dtype=np.int64)
    X = clustered_lattice(100, box_u, 7, 4000)
    w = catalogs.uniform_weights(X.shape[0], seed=9)
    sign = np.where(np.random.default_rng(10).random(len(w)) < 0.5, -1.0, 1.0)
    w = (w * sign).astype(np.float32)
    ref_c, ref_w = bf.count3(X, box_u, edges_u, w)
    assert np.any(ref_w < 0) and np.any(ref_w > 0)
    c, ws = oracle.Graph(X, box_u, edges_u, nthreads=2).count_3pcf(w)
    assert np.array_equal(c, ref_c)
    assert np.array_equal(ws, ref_w)


def wide_weights(n, seed, span_log2=20):
    """FP32 weights whose magnitudes span 2^span_log2 (log-uniform), both signs."""
    rng = np.random.default_rng(seed)
    mag = np.exp2(rng.uniform(-span_log2 / 2, span_log2 / 2, size=n)) * rng.uniform(0.5, 1.5, n)
    return (mag * np.where(rng.random(n) < 0.3, -1.0, 1.0)).astype(np.float32)


def test_3pcf_wide_weights_exact():
    """Weights spanning 2^20 (products beyond 128 bits): exact sums equal the
    rational all-triples sums bit for bit."""
    box_u = 30_000
    edges_u = np.array([0, 2500, 5000, 7000], dtype=np.int64)
    X = clustered_lattice(100, box_u, 17, 4000)
    w = wide_weights(X.shape[0], seed=18)
    assert np.abs(w).max() / np.abs(w).min() > 2 ** 18
    ref_c, ref_w = bf.count3(X, box_u, edges_u, w)
    c, ws = oracle.Graph(X, box_u, edges_u, nthreads=2).count_3pcf(w)
    assert np.array_equal(c, ref_c) and np.array_equal(ws, ref_w)


def test_4pcf_wide_weights_exact():
    box_u = 20_000
    edges_u = np.array([0, 2000, 4000], dtype=np.int64)
    X = clustered_lattice(60, box_u, 23, 2500)
    w = wide_weights(X.shape[0], seed=24)
    e_ref, o_ref, we_ref, wo_ref = bf.count4(X, box_u, edges_u, w)
    e, o, we, wo = oracle.Graph(X, box_u, edges_u).count_4pcf(w)
    assert np.array_equal(e, e_ref) and np.array_equal(o, o_ref)
    assert np.array_equal(we, we_ref) and np.array_equal(wo, wo_ref)


def test_3pcf_poisson_closed_form():
    """Unbinned triangle total of a uniform periodic catalogue.

    E[T] = C(N,3) p^2 * 15/32 with p = 4 pi R^3 / (3 L^3): two points
    uniform in a ball of radius R lie within R of each other with
    probability 15/32. Checked over 8 seeds at 4 sigma of their scatter.
    """
    L, R, N = 100.0, 10.0, 4000
    box_u = int(L * 1024)
    edges_u = np.array([0, int(R * 1024)], dtype=np.int64)
    totals = []
    for seed in range(8):
        X = oracle.quantize(catalogs.uniform(N, L, seed=100 + seed), box_u, True)
        totals.append(int(oracle.Graph(X, box_u, edges_u).count_3pcf().sum()))
    p = 4 * math.pi * (R * 1024) ** 3 / 3 / box_u ** 3
    expect = math.comb(N, 3) * p * p * 15 / 32
    mean, sd = np.mean(totals), np.std(totals, ddof=1)
    assert abs(mean - expect) < 4 * sd / math.sqrt(len(totals)) + 1e-3 * expect


# --------------------------------------------------------------------------
# a4 / a5: tetrahedra and parity


@pytest.mark.parametrize("periodic,seed", [(True, 11), (False, 12)])
def test_4pcf_matches_cliques(periodic, seed):
    box_u = 20_000
    edges_u = np.array([0, 1800, 3000, 4200], dtype=np.int64)
    X = np.concatenate([rand_lattice(50, box_u, seed), clustered_lattice(40, box_u, seed + 1, 2200)])
    bu = box_u if periodic else 0
    e_ref, o_ref = bf.count4(X, bu, edges_u)
    assert e_ref.sum() > 30 and np.abs(o_ref).sum() > 0
    g = oracle.Graph(X, bu, edges_u, nthreads=2)
    e, o = g.count_4pcf()
    assert np.array_equal(e, e_ref)
    assert np.array_equal(o, o_ref)


def test_4pcf_weighted_exact():
    box_u = 20_000
    edges_u = np.array([0, 2000, 4000], dtype=np.int64)
    X = clustered_lattice(60, box_u, 21, 2500)
    w = catalogs.uniform_weights(X.shape[0], seed=22)
    e_ref, o_ref, we_ref, wo_ref = bf.count4(X, box_u, edges_u, w)
    g = oracle.Graph(X, box_u, edges_u)
    e, o, we, wo = g.count_4pcf(w)
    assert np.array_equal(e, e_ref) and np.array_equal(o, o_ref)
    assert np.array_equal(we, we_ref) and np.array_equal(wo, wo_ref)
    _, _, we2, _ = g.count_4pcf(2 * w)
    assert np.array_equal(we2, 16 * we)


def _transform(X, box_u, fn):
    return np.mod(fn(X.astype(np.int64)), box_u).astype(np.int32)


def test_parity_mirror_rotation_relabel():
    box_u = 24_000
    edges_u = np.array([0, 1500, 2600, 3700, 4800, 5900], dtype=np.int64)
    X = np.concatenate([rand_lattice(250, box_u, 31), clustered_lattice(250, box_u, 32, 3000)])
    e0, o0 = oracle.Graph(X, box_u, edges_u).count_4pcf()
    assert np.abs(o0).sum() > 0
    # mirror x -> -x negates the odd channel exactly
    Xm = _transform(X, box_u, lambda x: x * np.array([-1, 1, 1]))
    em, om = oracle.Graph(Xm, box_u, edges_u).count_4pcf()
    assert np.array_equal(em, e0) and np.array_equal(om, -o0)
    # a proper 90-degree rotation keeps both channels
    Xr = _transform(X, box_u, lambda x: x[:, [1, 0, 2]] * np.array([-1, 1, 1]))
    er, orr = oracle.Graph(Xr, box_u, edges_u).count_4pcf()
    assert np.array_equal(er, e0) and np.array_equal(orr, o0)
    # relabelling the points changes nothing
    perm = np.random.default_rng(5).permutation(X.shape[0])
    ep, op = oracle.Graph(X[perm], box_u, edges_u).count_4pcf()
    assert np.array_equal(ep, e0) and np.array_equal(op, o0)
    # the 3pCF is mirror invariant too
    g0 = oracle.Graph(X, box_u, edges_u)
    assert np.array_equal(oracle.Graph(Xm, box_u, edges_u).count_3pcf(), g0.count_3pcf())


@pytest.mark.parametrize("mirrored_fraction", [0.0, 0.3, 0.5])
def test_parity_injection(mirrored_fraction):
    """Sec. 4.9: isolated chiral tetrahedra give odd = N_L - N_R exactly."""
    gold = load_golden("injection_tetrahedron.json")
    edges_u = np.array(gold["edges_u"], dtype=np.int64)
    n = gold["n_struct"]
    _, lat, mirrored = catalogs.lattice_tetrahedra(np.array(gold["shape_u"]), n, mirrored_fraction,
                                                   gold["box_u"], int(edges_u[-1]) + 1, seed=77)
    g = oracle.Graph(lat.astype(np.int32), gold["box_u"], edges_u)
    even, odd = g.count_4pcf()
    nb = len(edges_u) - 1
    reps = [oracle.config_bins(4, nb, k) for k in range(oracle.num_configs(4, nb))]
    k = [r for r, _ in reps].index(tuple(gold["rep"]))
    assert reps[k][1]  # chiral
    n_left = int((~mirrored).sum())
    n_right = int(mirrored.sum())
    assert even[k] == n and even.sum() == n
    assert odd[k] == gold["left_sign"] * (n_left - n_right)
    assert np.count_nonzero(odd) == (0 if n_left == n_right else 1)
    # each isolated tetrahedron has 4 triangles and 6 pairs
    assert g.count_3pcf().sum() == 4 * n
    assert g.pairs().sum() == 6 * n


def test_regular_tetrahedra_single_orbit():
    """Regular lattice tetrahedra land in (b,b,b,b,b,b) with no odd signal."""
    a = 2000
    shape = np.array([[0, 0, 0], [a, a, 0], [a, 0, a], [0, a, a]])
    edges_u = np.array([0, 1000, 2000, 3000, 4000], dtype=np.int64)
    box_u = 200_000
    _, lat, _ = catalogs.lattice_tetrahedra(shape, 60, 0.5, box_u, int(edges_u[-1]) + 1, seed=3)
    even, odd = oracle.Graph(lat.astype(np.int32), box_u, edges_u).count_4pcf()
    side = int(math.isqrt(2 * a * a))  # 2828: bin 2
    b = int(np.searchsorted(edges_u, side, side="right") - 1)
    k = [oracle.config_bins(4, 4, i)[0] for i in range(oracle.num_configs(4, 4))].index((b,) * 6)
    assert even[k] == 60 and even.sum() == 60 and not odd.any()


# --------------------------------------------------------------------------
# configurations


def test_config_counts_golden():
    gold = load_golden("config_counts.json")
    for nb, n in gold["3pcf"].items():
        assert oracle.num_configs(3, int(nb)) == n == math.comb(int(nb) + 2, 3)
    for nb, n in gold["4pcf"].items():
        k = int(nb)
        assert oracle.num_configs(4, k) == n == (k ** 6 + 9 * k ** 4 + 14 * k ** 2) // 24
    for nb, n in gold["4pcf_chiral"].items():
        k = int(nb)
        got = sum(oracle.config_bins(4, k, i)[1] for i in range(oracle.num_configs(4, k)))
        assert got == n == (k ** 6 - 3 * k ** 4 + 2 * k ** 2) // 24


def test_config_order_lexicographic():
    reps3 = [oracle.config_bins(3, 5, i)[0] for i in range(oracle.num_configs(3, 5))]
    assert reps3 == sorted(t for t in itertools.product(range(5), repeat=3) if t[0] <= t[1] <= t[2])
    ref4 = bf.configs4(3)
    reps4 = [oracle.config_bins(4, 3, i) for i in range(oracle.num_configs(4, 3))]
    assert [r for r, _ in reps4] == sorted(ref4)
    assert [c for _, c in reps4] == [ref4[r][1] for r in sorted(ref4)]


def test_cayley_menger_178():
    """Sec. 5.2: 178 of the 276 four-bin configurations are realisable."""
    gold = load_golden("config_counts.json")["cayley_menger"]
    centres = gold["centres_mpc"]
    slots = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    good = 0
    for k in range(oracle.num_configs(4, gold["nb"])):
        rep, _ = oracle.config_bins(4, gold["nb"], k)
        M = np.ones((5, 5))
        M[0, 0] = 0.0
        for a in range(4):
            M[a + 1, a + 1] = 0.0
        for s, (a, b) in enumerate(slots):
            M[a + 1, b + 1] = M[b + 1, a + 1] = centres[rep[s]] ** 2
        good += np.linalg.det(M) > 0
    assert good == gold["realisable"]


# --------------------------------------------------------------------------
# a6: pairs and the disconnected term


@pytest.mark.parametrize("periodic", [True, False])
def test_pairs_match_all_pairs(periodic):
    box_u = 30_000
    edges_u = np.array([0, 1000, 2500, 4000, 7000], dtype=np.int64)
    X = np.concatenate([rand_lattice(200, box_u, 41), adversarial_points(box_u, edges_u)])
    w = catalogs.uniform_weights(X.shape[0], seed=42)
    bu = box_u if periodic else 0
    ref, wref = bf.pairs(X, bu, edges_u, w)
    g = oracle.Graph(X, bu, edges_u)
    p, wp = g.pairs(w)
    assert np.array_equal(p, ref)
    assert np.array_equal(wp, wref)


def test_disconnected_golden_two_bins():
    gold = load_golden("disc_two_bins.json")
    reps = [oracle.config_bins(4, 2, k) for k in range(oracle.num_configs(4, 2))]
    assert ["".join(map(str, r)) for r, _ in reps] == gold["reps"]
    assert [int(c) for _, c in reps] == gold["chiral"]
    box_u = 40_000
    edges_u = np.array([0, 2000, 4000], dtype=np.int64)
    X = rand_lattice(300, box_u, 51)
    g = oracle.Graph(X, box_u, edges_u)
    p = g.pairs().astype(np.float64)
    xi_t = np.array(gold["xi"])
    rr = p / (1.0 + xi_t)  # choose RR so that xi comes out as the golden values
    _, xi, z = g.disconnected(rr=rr)
    np.testing.assert_allclose(xi, xi_t, rtol=0, atol=1e-15)
    np.testing.assert_allclose(z, gold["zeta_disc"], rtol=0, atol=1e-14)


def test_disconnected_analytic_rr_and_invariance():
    box_u = 50_000
    edges_u = np.array([0, 2000, 3000, 4500], dtype=np.int64)
    N = 3000
    X = rand_lattice(N, box_u, 61)
    g = oracle.Graph(X, box_u, edges_u)
    p, xi, z = g.disconnected()
    vol = [4 * math.pi / 3 * (int(edges_u[b + 1]) ** 3 - int(edges_u[b]) ** 3) for b in range(3)]
    rr = np.array([N * (N - 1) / 2 * v / box_u ** 3 for v in vol])
    np.testing.assert_allclose(xi, p / rr - 1.0, rtol=1e-13, atol=1e-13)
    # uniform points: xi consistent with zero within Poisson scatter
    assert np.all(np.abs(xi) < 5 / np.sqrt(rr))
    # S4 invariance: evaluating Eq. (disc) on any relabelling gives the same value
    slots = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
    for k in range(0, oracle.num_configs(4, 3), 5):
        rep, _ = oracle.config_bins(4, 3, k)
        binof = {frozenset(s): rep[i] for i, s in enumerate(slots)}
        for pm in itertools.permutations(range(4)):
            t = [binof[frozenset((pm[a], pm[b]))] for a, b in slots]
            v = xi[t[0]] * xi[t[5]] + xi[t[1]] * xi[t[4]] + xi[t[2]] * xi[t[3]]
            assert abs(v - z[k]) <= 1e-15 * (1 + abs(v))
    # weighted with unit weights equals unweighted
    p1, xi1, z1 = g.disconnected(w=np.ones(N, np.float32))
    np.testing.assert_allclose(xi1, xi, rtol=1e-14, atol=1e-15)
