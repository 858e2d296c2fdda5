"""GPU parity of the anisotropic (mu-binned) 3pCF against the CPU oracle:
counts bit for bit, exact weighted sums bit for bit (both sides round the
exact sum once)."""
import numpy as np
import pytest

import catalogs
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gs():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2607_06604_gb300 as m
    return m


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def clustered(n, box_u, seed, spread=4000):
    rng = np.random.default_rng(seed)
    centres = rng.integers(0, box_u, size=(max(1, n // 40), 3))
    X = centres[rng.integers(0, len(centres), size=n)] + rng.integers(-spread, spread + 1,
                                                                    size=(n, 3))
    return np.mod(X, box_u).astype(np.int32)


@pytest.mark.parametrize("periodic,nmu,nb,seed", [(True, 4, 5, 1), (False, 10, 8, 2),
                                                  (True, 64, 3, 3), (True, 1, 6, 4)])
def test_mu_counts_and_sums_bit_exact(gs, torch_mod, periodic, nmu, nb, seed):
    box_u = 150_000
    # clustered and uniform points, and a row of points on a line (collinear
    # triangles) and in a plane z = const (mu = 1)
    line = np.array([[60_000 + 500 * k, 70_000, 80_000] for k in range(30)], dtype=np.int32)
    plane = np.array([[20_000 + 900 * a, 30_000 + 700 * b, 40_000] for a in range(8)
                      for b in range(8)], dtype=np.int32)
    X = np.concatenate([clustered(9000, box_u, seed),
                        np.random.default_rng(seed + 50).integers(0, box_u, size=(6000, 3))
                        .astype(np.int32), line, plane])
    edges = catalogs.bin_edges_u(0.0, 9.0, nb)
    bu = box_u if periodic else 0
    w = catalogs.uniform_weights(len(X), seed=seed + 7)
    w[::4] *= -1.0
    og = oracle.Graph(X, bu, edges)
    rc, rs = og.count_3pcf_mu(nmu, w)
    assert rc.sum() > 100_000 and rc[:, nmu].sum() > 100 and rc[:, nmu - 1].sum() > 1000
    g = gs.gs_build_graph(dev(torch_mod, X), bu, edges)
    c, s = gs.gs_count_3pcf_mu(g, nmu, dev(torch_mod, w))
    assert np.array_equal(c.cpu().numpy(), rc)
    assert np.array_equal(s.cpu().numpy(), rs)
    # unweighted, host arrays in and out
    gh = gs.gs_build_graph(X, bu, edges)
    assert np.array_equal(gs.gs_count_3pcf_mu(gh, nmu, like=X), rc)


def test_mu_hand_triangles(gs):
    box_u = 100_000
    edges = np.array([0, 2000, 4000, 6000], dtype=np.int64)
    P = np.array([50_000, 50_000, 50_000])
    cases = [([3000, 0, 0], [0, 3000, 0], 4, 3), ([3000, 0, 0], [0, 0, 3000], 4, 0),
             ([2500, 0, 0], [5000, 0, 0], 4, 4), ([0, 3000, 0], [1800, 0, -2400], 5, 3),
             ([0, 3000, 0], [1800, 0, -2400], 10, 6), ([0, 3000, 0], [3000, 0, -4001], 5, 2)]
    for j, k, nmu, want in cases:
        X = np.array([P, P + j, P + k], dtype=np.int32)
        c = gs.gs_count_3pcf_mu(gs.gs_build_graph(X, box_u, edges), nmu, like=X)
        assert c.sum() == 1 and c.sum(axis=0)[want] == 1, (j, k, nmu)


def test_mu_sums_to_3pcf_with_long_rows_windows_and_shards(gs, torch_mod):
    """A dense clump gives rows longer than the shared staging (global
    staging path); the sum over mu bins equals the 3pCF, and out-of-core
    windows and hub shards change nothing."""
    box_u = 200_000
    rng = np.random.default_rng(9)
    X = np.concatenate([rng.integers(0, box_u, size=(40_000, 3)),
                        100_000 + rng.integers(-1500, 1501, size=(5000, 3))]).astype(np.int32)
    edges = np.array([0, 1500, 3000, 4500, 6000], dtype=np.int64)
    g = gs.gs_build_graph(dev(torch_mod, X), box_u, edges)
    assert gs.gs_graph_info(g)["max_degree"] > 2048
    like = dev(torch_mod, np.zeros(1))
    c = gs.gs_count_3pcf_mu(g, 6, like=like).cpu().numpy()
    c3 = gs.gs_count_3pcf(g, like=like).cpu().numpy()
    assert c.sum() > 10**10 and np.array_equal(c.sum(axis=1), c3)
    gw = gs.gs_build_graph(dev(torch_mod, X), box_u, edges, force_windows=3)
    assert np.array_equal(gs.gs_count_3pcf_mu(gw, 6, like=like).cpu().numpy(), c)
    parts = [gs.gs_count_3pcf_mu(g, 6, like=like, shard=k, shards=3).cpu().numpy()
             for k in range(3)]
    assert np.array_equal(parts[0] + parts[1] + parts[2], c)


@pytest.mark.parametrize("n", [0, 1, 2, 3])
def test_mu_tiny_catalogues(gs, n):
    box_u = 50_000
    X = (np.arange(3 * n).reshape(n, 3) * 700 + 20_000).astype(np.int32)
    edges = np.array([0, 2000, 4000], dtype=np.int64)
    c = gs.gs_count_3pcf_mu(gs.gs_build_graph(X, box_u, edges), 3, like=X)
    want = oracle.Graph(X, box_u, edges).count_3pcf_mu(3) if n else np.zeros_like(c)
    assert np.array_equal(c, want)


def test_mu_errors(gs):
    box_u = 50_000
    X = np.array([[1, 2, 3], [10, 20, 30], [400, 500, 600]], dtype=np.int32)
    g = gs.gs_build_graph(X, box_u, np.array([0, 2000, 4000], dtype=np.int64))
    for bad in (0, 65):
        with pytest.raises(gs.GSError):
            gs.gs_count_3pcf_mu(g, bad, like=X)
