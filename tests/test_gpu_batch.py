"""Batched persistent launch: one kernel over many uneven catalogues gives
exactly the per-catalogue results (integer histograms; exact weighted sums)."""
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


def test_batch_equals_single_and_oracle(gs):
    import torch
    L = 90.0
    box_u = int(L * 1024)
    edges = catalogs.bin_edges_u(0.0, 9.0, 6)
    sizes = [0, 5, 3000, 12000, 800, 20000, 1]
    cats, graphs, ws = [], [], []
    for k, n in enumerate(sizes):
        pos = catalogs.neyman_scott(n, L, seed=200 + k, sigma=1.5) if n else np.zeros((0, 3))
        X = oracle.quantize(pos, box_u, True) if n else np.zeros((0, 3), np.int32)
        w = catalogs.uniform_weights(max(n, 1), seed=300 + k)[:n]
        cats.append((X, w))
        graphs.append(gs.gs_build_graph(X, box_u, edges))
        ws.append(torch.from_numpy(np.ascontiguousarray(w)).cuda() if n else
                  torch.zeros(1, dtype=torch.float32, device="cuda"))
    out = gs.gs_count_3pcf_batch(graphs, ws)
    for k, (X, w) in enumerate(cats):
        c, s = out[k]
        sc, ss = gs.gs_count_3pcf(graphs[k], ws[k])
        assert np.array_equal(c.cpu().numpy(), sc.cpu().numpy())
        assert np.array_equal(s.cpu().numpy(), ss.cpu().numpy())
        if X.shape[0] > 2:
            rc, rw = oracle.Graph(X, box_u, edges).count_3pcf(w)
            assert np.array_equal(c.cpu().numpy(), rc)
            assert np.array_equal(s.cpu().numpy(), rw)
    # exact weighted sums are identical in and out of a batch
    out_x = gs.gs_count_3pcf_batch(graphs, ws)
    for k in range(len(sizes)):
        assert np.array_equal(out_x[k][1].cpu().numpy(),
                              gs.gs_count_3pcf(graphs[k], ws[k])[1].cpu().numpy())
    # unweighted batch, host outputs
    out_u = gs.gs_count_3pcf_batch(graphs)
    for k in range(len(sizes)):
        assert np.array_equal(out_u[k][0], out[k][0].cpu().numpy())


def test_batch_rejects_mixed_bins(gs):
    X = np.zeros((10, 3), np.int32)
    g1 = gs.gs_build_graph(X, 100_000, [0, 100, 200])
    g2 = gs.gs_build_graph(X, 100_000, [0, 100, 200, 300])
    with pytest.raises(gs.GSError) as e:
        gs.gs_count_3pcf_batch([g1, g2])
    assert e.value.status == -1


def test_recorded_plan_replays_exactly(gs):
    import torch
    L = 90.0
    box_u = int(L * 1024)
    edges = catalogs.bin_edges_u(0.0, 9.0, 6)
    graphs, refs = [], []
    for k, n in enumerate([3000, 15000, 7000]):
        X = oracle.quantize(catalogs.neyman_scott(n, L, seed=600 + k, sigma=1.5), box_u, True)
        g = gs.gs_build_graph(X, box_u, edges)
        graphs.append(g)
        refs.append(gs.gs_count_3pcf(g))
    plan = gs.gs_plan(graphs)
    stream = torch.cuda.Stream()
    for _ in range(3):  # replays rewrite the outputs from zero
        plan.launch(stream)
        counts = plan.wait(stream)
        for c, r in zip(counts, refs):
            assert np.array_equal(c.cpu().numpy(), r)
    plan.close()


def test_autotuner_picks_a_variant_with_identical_counts(gs):
    L = 100.0
    box_u = int(L * 1024)
    edges = catalogs.bin_edges_u(0.0, 9.0, 6)
    X = oracle.quantize(catalogs.neyman_scott(20_000, L, seed=700, sigma=1.5), box_u, True)
    w = catalogs.uniform_weights(X.shape[0], seed=701)
    g = gs.gs_build_graph(X, box_u, edges)
    ref_c, ref_w = gs.gs_count_3pcf(g, w)
    best = gs.gs_tune_3pcf(g, w)
    assert best in (0, 2, 4, 6, 32, 34, 64, 96)
    c, ws = gs.gs_count_3pcf(g, w, variant=-1)
    assert np.array_equal(c, ref_c) and np.array_equal(ws, ref_w)
    assert gs.gs_tune_3pcf(g) in (0, 2, 4, 6, 32, 34, 64, 96)
    assert np.array_equal(gs.gs_count_3pcf(g, variant=-1), ref_c)
