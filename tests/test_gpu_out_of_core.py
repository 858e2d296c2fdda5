"""Out-of-core row windows (Sec. 3.5.3): a graph whose edges exceed the
device budget keeps them in pinned host memory and every query streams
hub windows with their halo rows. Results must be bit-identical to the
resident graph for every window count (the paper validated all kernels in
single-pass and chunked modes, Sec. 4.8)."""
import numpy as np
import pytest

import catalogs
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    import torch
    assert torch.cuda.is_available()
    import paper_2607_06604_gb300 as m
    return m


@pytest.fixture(scope="module")
def case():
    L = 150.0
    box_u = int(L * 1024)
    pos = catalogs.neyman_scott(40_000, L, seed=91, sigma=2.0)
    X = oracle.quantize(pos, box_u, True)
    w = catalogs.uniform_weights(X.shape[0], seed=92)
    edges = catalogs.bin_edges_u(0.0, 10.0, 6)
    return X, box_u, edges, w


@pytest.fixture(scope="module")
def resident(gs, case):
    X, box_u, edges, w = case
    g = gs.gs_build_graph(X, box_u, edges)
    assert gs.gs_graph_info(g)["windows"] == 1
    out = {"c3": gs.gs_count_3pcf(g, w), "c3f": gs.gs_count_3pcf(g, w),
           "c4": gs.gs_count_4pcf_parity(g),
           "pairs": gs.gs_disconnected_4pcf(g, w), "export": gs.gs_graph_export(g),
           "info": gs.gs_graph_info(g)}
    # the resident path itself is pinned to the oracle: 3pCF counts and
    # exact weighted sums, 4pCF even and odd channels, weighted pair sums,
    # so every windowed result compared with it below is compared with the
    # oracle too
    og = oracle.Graph(X, box_u, edges)
    rc, rw = og.count_3pcf(w)
    assert np.array_equal(out["c3"][0], rc)
    assert np.array_equal(out["c3"][1], rw)
    re, ro = og.count_4pcf()
    assert re.sum() > 0 and np.array_equal(out["c4"][0], re) and np.array_equal(out["c4"][1], ro)
    rp, rxi, _ = og.disconnected(w)
    assert np.array_equal(out["pairs"][0], rp)
    np.testing.assert_allclose(out["pairs"][1], rxi, rtol=1e-12, atol=1e-12)
    return out


@pytest.mark.parametrize("windows", [1, 2, 3, 5, 8])
def test_forced_windows_bit_identical(gs, case, resident, windows):
    X, box_u, edges, w = case
    g = gs.gs_build_graph(X, box_u, edges, force_windows=windows)
    info = gs.gs_graph_info(g)
    assert info["windows"] == windows or (windows > 1 and info["windows"] > 1)
    c, ws = gs.gs_count_3pcf(g, w)
    assert np.array_equal(c, resident["c3"][0])
    assert np.array_equal(ws, resident["c3"][1])  # exact sums: bit-identical
    _, wf = gs.gs_count_3pcf(g, w)
    assert np.array_equal(wf, resident["c3f"][1])
    e, o = gs.gs_count_4pcf_parity(g)
    assert np.array_equal(e, resident["c4"][0]) and np.array_equal(o, resident["c4"][1])
    p, xi, z = gs.gs_disconnected_4pcf(g, w)
    assert np.array_equal(p, resident["pairs"][0])
    assert np.array_equal(xi, resident["pairs"][1]) and np.array_equal(z, resident["pairs"][2])
    ex = gs.gs_graph_export(g)
    for a, b in zip(ex, resident["export"]):
        assert np.array_equal(a, b)
    for k in ("edges", "probe_words", "walk_words", "max_degree", "edge_slots"):
        assert info[k] == resident["info"][k], k


def test_budget_driven_windows(gs, case, resident):
    X, box_u, edges, w = case
    slots = resident["info"]["edge_slots"]
    # two window buffers of 40% of the edges each: own rows plus the next
    # x-slab plus the wrap-around slab fit, the whole graph does not
    budget = int(slots * 4 * 0.8)
    g = gs.gs_build_graph(X, box_u, edges, budget=budget)
    info = gs.gs_graph_info(g)
    assert info["windows"] >= 2
    c, ws = gs.gs_count_3pcf(g, w)
    assert np.array_equal(c, resident["c3"][0]) and np.array_equal(ws, resident["c3"][1])
    # a query may ask for smaller windows than the build did
    c2 = gs.gs_count_3pcf(g, budget=int(budget * 0.75))
    assert np.array_equal(c2, resident["c3"][0])
    e, o = gs.gs_count_4pcf_parity(g)
    assert np.array_equal(e, resident["c4"][0]) and np.array_equal(o, resident["c4"][1])


def test_budget_too_small(gs, case):
    X, box_u, edges, _ = case
    with pytest.raises(gs.GSError) as e:
        gs.gs_build_graph(X, box_u, edges, budget=4096)
    assert e.value.status == -3
    # the library stays usable after the error
    g = gs.gs_build_graph(X[:1000], box_u, edges)
    assert gs.gs_count_3pcf(g).sum() >= 0


@pytest.mark.parametrize("shards,windows", [(2, 0), (3, 0), (4, 3)])
def test_hub_shards_sum_exactly(gs, case, resident, shards, windows):
    """Hub shards (the multi-GPU split of one catalogue) run one after
    another on this GPU; their counts add up to the unsharded result."""
    X, box_u, edges, w = case
    g = gs.gs_build_graph(X, box_u, edges, force_windows=windows)
    c3 = sum(gs.gs_count_3pcf(g, shard=k, shards=shards).astype(np.int64) for k in range(shards))
    assert np.array_equal(c3, resident["c3"][0].astype(np.int64))
    e = np.zeros_like(resident["c4"][0], dtype=np.int64)
    o = np.zeros_like(resident["c4"][1])
    p = np.zeros(len(edges) - 1, dtype=np.int64)
    for k in range(shards):
        ek, ok = gs.gs_count_4pcf_parity(g, shard=k, shards=shards)
        e += ek.astype(np.int64)
        o += ok
        p += gs.gs_disconnected_4pcf(g, zeta=False, shard=k, shards=shards)[0].astype(np.int64)
    assert np.array_equal(e, resident["c4"][0].astype(np.int64))
    assert np.array_equal(o, resident["c4"][1])
    assert np.array_equal(p, resident["pairs"][0].astype(np.int64))
    # each shard rounds its exact sum once; the FP64 sum of those rounded
    # values is within a few ulps of the whole graph's single rounding
    ws = sum(gs.gs_count_3pcf(g, w, shard=k, shards=shards)[1] for k in range(shards))
    np.testing.assert_allclose(ws, resident["c3"][1], rtol=1e-13)
