"""Pins of the oracle's signed-weight connected 4pCF (Sec. 3.3)."""
import json
import os

import numpy as np

import catalogs
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_signed_pair_sum_is_the_landy_szalay_numerator():
    """With data weights w_D and random weights w_R on D u R, the signed pair
    sum is DD w_D^2 + DR w_D w_R + RR w_R^2 (Sec. 3.3), with DD, DR, RR counted
    separately (DR = pairs of the union minus DD minus RR)."""
    box_u = 60_000
    edges = np.array([0, 2000, 4000, 6000], dtype=np.int64)
    rng = np.random.default_rng(3)
    D = rng.integers(0, box_u, size=(700, 3)).astype(np.int32)
    R = rng.integers(0, box_u, size=(1500, 3)).astype(np.int32)
    U = np.concatenate([D, R])
    wD = np.float32(1.0 / len(D))
    wR = np.float32(-1.0 / len(R))
    w = np.concatenate([np.full(len(D), wD, np.float32), np.full(len(R), wR, np.float32)])
    gU = oracle.Graph(U, box_u, edges)
    DD = oracle.Graph(D, box_u, edges).pairs().astype(np.float64)
    RR = oracle.Graph(R, box_u, edges).pairs().astype(np.float64)
    DR = gU.pairs().astype(np.float64) - DD - RR
    _, signed = gU.pairs(w)
    expect = DD * float(wD) ** 2 + DR * float(wD) * float(wR) + RR * float(wR) ** 2
    np.testing.assert_allclose(signed, expect, rtol=1e-14, atol=1e-18)
    # xi of the estimator is that numerator over the randoms' pair sum
    gR = oracle.Graph(R, box_u, edges)
    out = oracle.connected_4pcf(gU, w, gR, np.full(len(R), np.float32(1.0 / len(R))))
    _, rr = gR.pairs(np.full(len(R), np.float32(1.0 / len(R))))
    np.testing.assert_allclose(out["xi"], signed / rr, rtol=1e-15)


def test_connected_injection_count_level():
    """Sec. 4.9 with the signed-weight estimator: isolated chiral tetrahedra
    as data, randoms in a cube farther than r_max from every structure. No
    quadruplet mixes the two, so the signed odd sum at the injected orbit is
    w_D^4 (N_L - N_R) plus w_R^4 times the randoms' own odd count, and the
    estimator divides it by the randoms' weighted even count."""
    gold = json.load(open(os.path.join(GOLDEN, "injection_tetrahedron.json")))
    edges = np.array(gold["edges_u"], dtype=np.int64)
    rmax = int(edges[-1])
    n = 200
    box_u = 2 * gold["box_u"]
    _, lat, mirrored = catalogs.lattice_tetrahedra(np.array(gold["shape_u"]), n, 0.3,
                                                   gold["box_u"], rmax + 1, seed=5)
    assert lat[:, 0].max() < gold["box_u"]
    rng = np.random.default_rng(8)
    R = rng.integers(0, 24_000, size=(1500, 3))
    R[:, 0] += gold["box_u"] + 2 * rmax
    U = np.concatenate([lat, R]).astype(np.int32)
    nD, nR = lat.shape[0], R.shape[0]
    wD, wR = np.float32(1.0 / nD), np.float32(-1.0 / nR)
    wr = np.float32(1.0 / nR)
    w = np.concatenate([np.full(nD, wD, np.float32), np.full(nR, wR, np.float32)])
    gU = oracle.Graph(U, box_u, edges)
    gR = oracle.Graph(R.astype(np.int32), box_u, edges)
    out = oracle.connected_4pcf(gU, w, gR, np.full(nR, wr))
    r_even, r_odd = gR.count_4pcf()
    nb = len(edges) - 1
    reps = [oracle.config_bins(4, nb, i)[0] for i in range(oracle.num_configs(4, nb))]
    k = reps.index(tuple(gold["rep"]))
    assert r_even[k] > 0
    nl, nr = int((~mirrored).sum()), int(mirrored.sum())
    f = float
    pred = f(wD) ** 4 * gold["left_sign"] * (nl - nr) + f(wR) ** 4 * f(r_odd[k])
    np.testing.assert_allclose(out["zeta_odd"][k], pred / (f(wr) ** 4 * f(r_even[k])),
                               rtol=1e-12)
    # every orbit: data tetrahedra sit only at the injected orbit
    keep = r_even > 0
    d_even = np.zeros(len(reps))
    d_even[k] = n
    pe = (f(wD) ** 4 * d_even + f(wR) ** 4 * r_even.astype(np.float64))[keep]
    np.testing.assert_allclose(out["zeta_even"][keep], pe / (f(wr) ** 4 * r_even[keep]),
                               rtol=1e-12)
    np.testing.assert_array_equal(out["zeta_conn"], out["zeta_even"] - out["zeta_disc"])
