"""Configuration tooling on the GPU against the oracle: Cayley-Menger mask
(Sec. 5.2) and exact rebinning (Sec. 5.1)."""
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


def test_cm_mask_printed_count(gs):
    edges = np.array([int(20 * 1024 + b * 11.25 * 1024) for b in range(5)], dtype=np.int64)
    mask, kept = gs.gs_config_mask_cm(4, edges)
    assert kept == 178 and int(mask.sum()) == 178 and len(mask) == 276
    assert np.array_equal(mask, oracle.config_mask_cm(4, edges))


@pytest.mark.parametrize("nb,seed", [(1, 1), (2, 2), (3, 3), (5, 5), (6, 6)])
def test_cm_mask_random_edges(gs, nb, seed):
    rng = np.random.default_rng(seed)
    edges = np.cumsum(np.concatenate([[rng.integers(0, 30_000)],
                                      rng.integers(1, 40_000, size=nb)])).astype(np.int64)
    mask, kept = gs.gs_config_mask_cm(nb, edges)
    want = oracle.config_mask_cm(nb, edges)
    assert np.array_equal(mask, want) and kept == int(want.sum())


def test_cm_mask_errors(gs):
    with pytest.raises(gs.GSError) as e:
        gs.gs_config_mask_cm(2, np.array([0, 5, 5], dtype=np.int64))
    assert e.value.status == -1
    with pytest.raises(gs.GSError) as e:
        gs.gs_config_mask_cm(2, np.array([0, 5, (1 << 19) + 1], dtype=np.int64))
    assert e.value.status == -2


def random_counts4(nb, seed, weighted):
    rng = np.random.default_rng(seed)
    n = oracle.num_configs(4, nb)
    chiral = np.array([oracle.config_bins(4, nb, c)[1] for c in range(n)])
    e = rng.integers(0, 1 << 40, n).astype(np.uint64)
    o = rng.integers(-(1 << 30), 1 << 30, n)
    o[~chiral] = 0
    we = rng.standard_normal(n) if weighted else None
    wo = np.where(chiral, rng.standard_normal(n), 0.0) if weighted else None
    return e, o, we, wo


@pytest.mark.parametrize("nbf,nbc,bmap", [
    (6, 3, [0, 0, 1, 1, 2, 2]), (8, 4, [-1, 0, 0, 1, 1, 2, 3, -1]), (5, 5, [4, 3, 2, 1, 0]),
    (4, 1, [0, 0, 0, 0]), (3, 2, [-1, -1, -1])])
def test_rebin_4pcf_matches_oracle(gs, nbf, nbc, bmap):
    e, o, we, wo = random_counts4(nbf, nbf * 10 + nbc, True)
    bmap = np.array(bmap, dtype=np.int32)
    want = oracle.rebin_4pcf(nbf, nbc, bmap, e, o, we, wo)
    got = gs.gs_rebin_4pcf(nbf, nbc, bmap, e, o, we, wo)
    for g_, w_ in zip(got, want):
        assert np.array_equal(g_, w_)  # same order of FP64 additions: bit-identical


@pytest.mark.parametrize("nbf,nbc", [(12, 4), (60, 20), (30, 30)])
def test_rebin_3pcf_matches_oracle(gs, nbf, nbc):
    rng = np.random.default_rng(nbf)
    n = oracle.num_configs(3, nbf)
    c = rng.integers(0, 1 << 40, n).astype(np.uint64)
    w = rng.standard_normal(n)
    bmap = np.minimum(np.arange(nbf) * nbc // nbf, nbc - 1).astype(np.int32)
    bmap[0] = -1
    wc, ww = oracle.rebin_3pcf(nbf, nbc, bmap, c, w)
    gc, gw = gs.gs_rebin_3pcf(nbf, nbc, bmap, c, w)
    assert np.array_equal(gc, wc) and np.array_equal(gw, ww)
    gc2, none = gs.gs_rebin_3pcf(nbf, nbc, bmap, counts=c)
    assert none is None and np.array_equal(gc2, wc)


def test_rebin_gpu_counts_equal_direct_coarse_counts(gs):
    """End to end on the GPU: fine counts rebinned equal the counts taken
    directly on the coarse edges (3pCF, and parity 4pCF with odd)."""
    import torch
    L = 90.0
    box_u = int(L * 1024)
    X = oracle.quantize(catalogs.neyman_scott(9000, L, seed=311, sigma=1.5), box_u, True)
    w = catalogs.uniform_weights(len(X), seed=312)
    fine = np.array([int(700 * k) for k in range(13)], dtype=np.int64)
    coarse = fine[2:11:2]
    bmap = np.full(12, -1, dtype=np.int32)
    bmap[2:10] = np.arange(8) // 2
    gf = gs.gs_build_graph(X, box_u, fine)
    gc = gs.gs_build_graph(X, box_u, coarse)
    fc, fw = gs.gs_count_3pcf(gf, w)
    cc, cw = gs.gs_count_3pcf(gc, w)
    rc, rw = gs.gs_rebin_3pcf(12, 4, bmap, fc, fw)
    assert cc.sum() > 100_000 and np.array_equal(rc, cc)
    np.testing.assert_allclose(rw, cw, rtol=1e-12)
    fine4 = fine[:7]
    coarse4 = fine[1:6:2]
    bmap4 = np.array([-1, 0, 0, 1, 1, -1], dtype=np.int32)
    fe, fo = gs.gs_count_4pcf_parity(gs.gs_build_graph(X, box_u, fine4))
    ce, co = gs.gs_count_4pcf_parity(gs.gs_build_graph(X, box_u, coarse4))
    re, ro, _, _ = gs.gs_rebin_4pcf(6, 2, bmap4, fe, fo)
    assert ce.sum() > 10_000 and np.abs(co).sum() > 0
    assert np.array_equal(re, ce) and np.array_equal(ro, co)
    # device arrays in and out
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    de, do_, _, _ = gs.gs_rebin_4pcf(6, 2, dev(bmap4), dev(fe), dev(fo))
    assert de.is_cuda and np.array_equal(de.cpu().numpy(), ce) and np.array_equal(do_.cpu().numpy(), co)


def test_rebin_errors(gs):
    with pytest.raises(gs.GSError) as e:
        gs.gs_rebin_3pcf(3, 2, np.array([0, 2, 1], np.int32), np.zeros(10, np.uint64))
    assert e.value.status == -1
    with pytest.raises(gs.GSError) as e:
        gs.gs_rebin_4pcf(17, 2, np.zeros(17, np.int32), np.zeros(1, np.uint64))
    assert e.value.status == -2


def diagonal(nb):
    idx = {oracle.config_bins(3, nb, k)[0]: k for k in range(oracle.num_configs(3, nb))}
    return [idx[(b, b, b)] for b in range(nb)]


@pytest.mark.parametrize("periodic", [True, False])
def test_equilateral_matches_oracle_and_full_3pcf(gs, periodic):
    L = 150.0
    box_u = int(L * 1024)
    X = oracle.quantize(catalogs.neyman_scott(40_000, L, seed=321, sigma=2.0, periodic=periodic),
                        box_u, periodic)
    w = catalogs.uniform_weights(len(X), seed=322)
    edges = catalogs.bin_edges_u(0.0, 10.0, 7)
    bu = box_u if periodic else 0
    c, ws = oracle.equilateral_3pcf(oracle.Graph(X, bu, edges), w)
    g = gs.gs_build_graph(X, bu, edges)
    gc, gw = gs.gs_count_3pcf_equilateral(g, w)
    assert c.sum() > 100_000
    assert np.array_equal(gc, c)
    assert np.array_equal(gw, ws)
    fc, fw = gs.gs_count_3pcf(g, w)
    sel = diagonal(len(edges) - 1)
    assert np.array_equal(gc, fc[sel]) and np.array_equal(gw, fw[sel])
    assert np.array_equal(gs.gs_count_3pcf_equilateral(g), c)
    # the merge-walk's instantiation (512) and every launch path of it: hash
    # of the hub row (1), hub rows from global memory (2), a 2 KB table (8),
    # compacted weighted hits (32), prefetch ring (64)
    for v in (512, 513, 514, 520, 544, 576, 584):
        vc, vw = gs.gs_count_3pcf_equilateral(g, w, variant=v)
        assert np.array_equal(vc, c), v
        assert np.array_equal(vw, gw), v
    # out-of-core windows and hub shards
    g3 = gs.gs_build_graph(X, bu, edges, force_windows=3)
    c3, w3 = gs.gs_count_3pcf_equilateral(g3, w)
    assert np.array_equal(c3, gc) and np.array_equal(w3, gw)
    cs = sum(gs.gs_count_3pcf_equilateral(g, shard=k, shards=2).astype(np.int64) for k in range(2))
    assert np.array_equal(cs, gc.astype(np.int64))


def test_equilateral_long_rows(gs):
    """A dense clump gives hub rows longer than the staged capacity (4096
    words), which are searched in global memory."""
    import torch
    rng = np.random.default_rng(331)
    box_u = 200_000
    X = np.concatenate([rng.integers(90_000, 94_000, size=(4600, 3)),
                        rng.integers(0, box_u, size=(20_000, 3))]).astype(np.int32)
    edges = np.array([0, 2500, 4500, 7000], dtype=np.int64)
    g = gs.gs_build_graph(X, box_u, edges)
    assert gs.gs_graph_info(g)["max_degree"] > 4096
    fc = gs.gs_count_3pcf(g)
    gc = gs.gs_count_3pcf_equilateral(g)
    assert np.array_equal(gc, fc[diagonal(3)]) and gc.sum() > 0
    assert np.array_equal(gs.gs_count_3pcf_equilateral(g, variant=512), gc)
    Xd = torch.from_numpy(X).cuda()
    gd = gs.gs_count_3pcf_equilateral(gs.gs_build_graph(Xd, box_u, edges), like=Xd)
    assert gd.is_cuda and np.array_equal(gd.cpu().numpy(), gc)
