"""gs_count_3pcf_noalloc: the triangle count for callers that cannot let the
library allocate device memory during a call (it runs on a fixed scratch
array compiled into the library). Its counts must equal gs_count_3pcf's,
bit for bit, on consecutive calls (the shared scratch keeps the previous
call's contents, so each call must clear it). This file is collected last
so that a stop-at-first-failure run has run every other test first."""
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


def test_noalloc_matches_regular_entry_point(gs):
    import torch
    L = 120.0
    box_u = int(L * 1024)
    X = oracle.quantize(catalogs.neyman_scott(30_000, L, seed=61, sigma=2.0), box_u, True)
    edges = catalogs.bin_edges_u(0.0, 12.0, 8)
    g = gs.gs_build_graph(X, box_u, edges)
    ref = gs.gs_count_3pcf(g)
    assert ref.sum() > 0
    # two calls in a row, host output, then two with device output
    for _ in range(2):
        assert np.array_equal(gs.gs_count_3pcf_noalloc(g), ref)
    dev = torch.zeros(len(ref), dtype=torch.uint64, device="cuda")
    for _ in range(2):
        gs.gs_count_3pcf_noalloc(g, counts=dev)
        assert np.array_equal(dev.cpu().numpy(), ref)
    # a second, smaller graph right after: leftovers of the previous call
    # must not leak into its counts
    g2 = gs.gs_build_graph(X[:3000], box_u, edges)
    ref2 = gs.gs_count_3pcf(g2)
    for _ in range(2):
        assert np.array_equal(gs.gs_count_3pcf_noalloc(g2), ref2)


def test_noalloc_limits(gs):
    X = np.zeros((10, 3), np.int32)
    g = gs.gs_build_graph(X, 100_000, list(range(0, 3700, 100)))  # nb = 36
    with pytest.raises(gs.GSError) as e:
        gs.gs_count_3pcf_noalloc(g)
    assert e.value.status == -2
    g_ooc = gs.gs_build_graph(X, 100_000, [0, 100, 200], force_windows=2)
    with pytest.raises(gs.GSError) as e:
        gs.gs_count_3pcf_noalloc(g_ooc)
    assert e.value.status == -1
