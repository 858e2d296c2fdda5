"""GPU parity of the pixelised-direction parity 4pCF (Sec. 3.2's pixel byte
per spoke and the |V| < 1e-9 degenerate rule) through the C ABI against the
oracle: the direction pixels bit for bit, even and odd channels bit for bit
on clustered periodic and open catalogues, with weights (exact sums), on
the global-workspace path, with coincident points, and the injection test."""
import json
import os

import numpy as np
import pytest

import catalogs
import oracle

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def gs():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2607_06604_gb300 as m
    return m


def test_direction_pixels_bit_exact(gs):
    import torch
    rng = np.random.default_rng(11)
    d = np.concatenate([rng.integers(-600_000, 600_001, size=(200_000, 3)),
                        rng.integers(-3, 4, size=(2000, 3)),
                        np.array([[12, 5, 0], [99, 41, 7], [-70, 29, -3], [1, 1, 0], [0, 0, 5],
                                  [0, 0, -5], [-4, 0, 0], [0, -4, 1], [3, -3, 3]])])
    # directions within a fraction of a lattice unit of a sector edge (Pell
    # approximations of tan(pi/8) = sqrt 2 - 1 and tan(3 pi/8) = sqrt 2 + 1,
    # in every quadrant) and components up to the documented 2^20
    pell = [(5, 2), (12, 5), (29, 12), (70, 29), (169, 70), (408, 169), (985, 408),
            (2378, 985), (5741, 2378), (13860, 5741), (33461, 13860), (80782, 33461),
            (195025, 80782), (470832, 195025)]
    edge = []
    for a_, b_ in pell:
        for sx, sy in ((1, 1), (-1, 1), (-1, -1), (1, -1)):
            for z_ in (0, 7, -11):
                edge += [[sx * a_, sy * b_, z_], [sx * b_, sy * a_, z_]]
    big = rng.integers(-(1 << 20) + 1, 1 << 20, size=(20_000, 3))
    d = np.concatenate([d, np.array(edge), big])
    d = d[np.any(d != 0, axis=1)].astype(np.int32)
    ref = oracle.direction_pixels(d)
    assert np.array_equal(gs.gs_direction_pixels(d), ref)
    got = gs.gs_direction_pixels(torch.from_numpy(d).cuda())
    assert np.array_equal(got.cpu().numpy(), ref)


@pytest.mark.parametrize("periodic,nb,seed", [(True, 4, 141), (False, 6, 142), (True, 8, 143)])
def test_pixel_parity_clustered(gs, periodic, nb, seed):
    L = 100.0
    box_u = int(L * 1024)
    pos = catalogs.neyman_scott(12_000, L, seed=seed, sigma=1.5, periodic=periodic)
    X = oracle.quantize(pos, box_u, periodic)
    edges = catalogs.bin_edges_u(0.0, 9.0, nb)
    bu = box_u if periodic else 0
    og = oracle.Graph(X, bu, edges)
    re, ro = og.count_4pcf(pixel=True)
    ee, eo = og.count_4pcf()
    assert re.sum() > 100_000 and np.abs(ro).sum() > 0
    assert not np.array_equal(ro, eo)  # the pixelised channel is its own reading
    g = gs.gs_build_graph(X, bu, edges)
    for variant in (0, 1, 4):  # default, global workspace, binned by search
        ge, go = gs.gs_count_4pcf_parity_pix(g, variant=variant)
        assert np.array_equal(ge, re) and np.array_equal(go, ro), variant
    # the exact channel on the same graph is untouched
    xe, xo = gs.gs_count_4pcf_parity(g)
    assert np.array_equal(xe, ee) and np.array_equal(xo, eo)


def test_pixel_parity_weighted(gs):
    box_u = 80_000
    rng = np.random.default_rng(151)
    X = np.concatenate([rng.integers(0, box_u, size=(4000, 3)),
                        np.mod(40_000 + rng.integers(-5000, 5001, size=(300, 3)), box_u)])
    X = X.astype(np.int32)
    w = catalogs.uniform_weights(X.shape[0], seed=153)
    edges = np.array([0, 2500, 5000, 7000], dtype=np.int64)
    re, ro, rwe, rwo = oracle.Graph(X, box_u, edges).count_4pcf(w, pixel=True)
    g = gs.gs_build_graph(X, box_u, edges)
    ge, go, gwe, gwo = gs.gs_count_4pcf_parity_pix(g, w)
    assert np.array_equal(ge, re) and np.array_equal(go, ro)
    assert np.array_equal(gwe, rwe) and np.array_equal(gwo, rwo)


def test_pixel_parity_coincident_points(gs):
    """Coincident points (distance 0, bin 0) give spokes of zero length: such
    tetrahedra are degenerate in the pixelised channel on both sides."""
    box_u = 50_000
    rng = np.random.default_rng(161)
    base = np.mod(25_000 + rng.integers(-1500, 1501, size=(60, 3)), box_u)
    X = np.concatenate([base, base[:20], base[:5]]).astype(np.int32)
    edges = np.array([0, 800, 1600, 2400], dtype=np.int64)
    re, ro = oracle.Graph(X, box_u, edges).count_4pcf(pixel=True)
    g = gs.gs_build_graph(X, box_u, edges)
    ge, go = gs.gs_count_4pcf_parity_pix(g)
    assert re.sum() > 1000
    assert np.array_equal(ge, re) and np.array_equal(go, ro)


@pytest.mark.parametrize("mirrored_fraction", [0.0, 0.3])
def test_pixel_parity_injection_gpu(gs, mirrored_fraction):
    with open(os.path.join(GOLDEN, "injection_tetrahedron.json")) as f:
        gold = json.load(f)
    edges_u = np.array(gold["edges_u"], dtype=np.int64)
    n = gold["n_struct"]
    _, lat, mirrored = catalogs.lattice_tetrahedra(np.array(gold["shape_u"]), n, mirrored_fraction,
                                                   gold["box_u"], int(edges_u[-1]) + 1, seed=79)
    g = gs.gs_build_graph(lat.astype(np.int32), gold["box_u"], edges_u)
    even, odd = gs.gs_count_4pcf_parity_pix(g)
    nb = len(edges_u) - 1
    k = [gs.gs_config_bins(4, nb, i)[0] for i in range(gs.gs_num_configs(4, nb))].index(
        tuple(gold["rep"]))
    n_left, n_right = int((~mirrored).sum()), int(mirrored.sum())
    assert even[k] == n and even.sum() == n
    assert odd[k] == gold["left_sign"] * (n_left - n_right)
