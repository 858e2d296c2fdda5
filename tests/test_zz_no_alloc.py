"""gs_count_3pcf_noalloc: the triangle count for callers that cannot let the
library allocate device memory during a call (a process that has handed all
device memory to its own pool, or a real-time loop that must stay clear of
the allocator's locks and synchronisation). It runs on a fixed scratch
array compiled into the library. Its counts must equal gs_count_3pcf's and
the oracle's, bit for bit, on consecutive calls (the shared scratch keeps
the previous call's contents, so each call must clear it), for every launch
variant, with host and device outputs, at the largest bin count the scratch
holds, and on a graph whose longest row sends the counts straight to the
global histograms; and free device memory must not change across calls.
This file is collected last so that a stop-at-first-failure run has run
every other test first."""
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


def free_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def check_calls(gs, g, ref, **opts):
    """Two calls in a row with host output, then two with device output."""
    import torch
    for _ in range(2):
        assert np.array_equal(gs.gs_count_3pcf_noalloc(g, **opts), ref), opts
    dev = torch.zeros(len(ref), dtype=torch.uint64, device="cuda")
    for _ in range(2):
        gs.gs_count_3pcf_noalloc(g, counts=dev, **opts)
        assert np.array_equal(dev.cpu().numpy(), ref), opts


def test_noalloc_matches_regular_entry_point_and_oracle(gs):
    import torch
    L = 120.0
    box_u = int(L * 1024)
    X = oracle.quantize(catalogs.neyman_scott(30_000, L, seed=61, sigma=2.0), box_u, True)
    edges = catalogs.bin_edges_u(0.0, 12.0, 8)
    g = gs.gs_build_graph(X, box_u, edges)
    ref = gs.gs_count_3pcf(g)
    assert ref.sum() > 0
    assert np.array_equal(ref, oracle.Graph(X, box_u, edges).count_3pcf())
    # every launch variant the entry point honours: hash path (1), hub rows
    # from global memory (2), computed configuration ranks (4), a 2 KB table
    # with split or hashed rows (8)
    for variant in (0, 1, 2, 4, 8):
        check_calls(gs, g, ref, variant=variant)
    # variant -1 takes the tuned choice, as gs_count_3pcf does
    gs.gs_tune_3pcf(g)
    check_calls(gs, g, ref, variant=-1)
    # no device memory is taken by the calls themselves (host and device
    # outputs; the output tensor is allocated before the first reading)
    out = torch.zeros(len(ref), dtype=torch.uint64, device="cuda")
    gs.gs_count_3pcf_noalloc(g, counts=out)
    before = free_bytes()
    for _ in range(3):
        host = gs.gs_count_3pcf_noalloc(g)
        gs.gs_count_3pcf_noalloc(g, counts=out)
    assert free_bytes() == before
    assert np.array_equal(host, ref) and np.array_equal(out.cpu().numpy(), ref)
    # a second, smaller graph right after: leftovers of the previous call
    # must not leak into its counts
    g2 = gs.gs_build_graph(X[:3000], box_u, edges)
    ref2 = gs.gs_count_3pcf(g2)
    assert np.array_equal(ref2, oracle.Graph(X[:3000], box_u, edges).count_3pcf())
    check_calls(gs, g2, ref2)


def test_noalloc_largest_bin_count(gs):
    """nb = 35 (C(37,3) = 7770 configurations, the most the scratch holds):
    the counts of the last configurations sit at the scratch array's end on
    their way to a host output."""
    L = 60.0
    box_u = int(L * 1024)
    X = oracle.quantize(catalogs.uniform(6000, L, seed=62), box_u, True)
    edges = catalogs.bin_edges_u(0.0, 14.0, 35)
    g = gs.gs_build_graph(X, box_u, edges)
    ref = gs.gs_count_3pcf(g)
    assert len(ref) == 7770 and ref[-1] > 0
    assert np.array_equal(ref, oracle.Graph(X, box_u, edges).count_3pcf())
    check_calls(gs, g, ref)


def test_noalloc_global_histogram_path(gs):
    """A hub with 66,000 forward neighbours (more than 65,535) sends every
    count straight to the 64-bit histograms in the scratch array. The hub
    sees two coincident clumps A (65,000 points) and B (1,000 points);
    points inside a clump are closer than the first bin edge, so the only
    triangles are hub-a-b, |A| |B| of them in one configuration."""
    box_u = 100_000
    edges = np.array([100, 2000, 4000], dtype=np.int64)
    hub = np.array([[9000, 10000, 10000]], dtype=np.int32)
    A = np.tile(np.array([[12500, 10000, 10000]], dtype=np.int32), (65_000, 1))
    B = np.tile(np.array([[12000, 11500, 10000]], dtype=np.int32), (1_000, 1))
    X = np.concatenate([hub, A, B])
    g = gs.gs_build_graph(X, box_u, edges)
    assert gs.gs_graph_info(g)["max_degree"] > 65535
    # hub-A 3500 (bin 1), hub-B 3354 (bin 1), A-B 1581 (bin 0)
    ref = np.zeros(gs.gs_num_configs(3, 2), dtype=np.uint64)
    ref[[k for k in range(len(ref)) if oracle.config_bins(3, 2, k)[0] == (0, 1, 1)][0]] = 65_000 * 1_000
    assert np.array_equal(gs.gs_count_3pcf(g), ref)
    check_calls(gs, g, ref)


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
