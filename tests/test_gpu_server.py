"""Request loop: requests of different sizes, kinds and bin counts submitted
together (and under a tight memory budget) give exactly what each gives
alone through the single-call API."""
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


def make_requests():
    L = 100.0
    box_u = int(L * 1024)
    reqs = []
    for k, n in enumerate([4000, 12000, 700, 20000, 2500, 9000, 0, 15000]):
        pos = catalogs.neyman_scott(max(n, 1), L, seed=400 + k, sigma=1.5)[:n]
        X = oracle.quantize(pos, box_u, True) if n else np.zeros((0, 3), np.int32)
        nb = 6 if k % 3 else 4
        edges = catalogs.bin_edges_u(0.0, 8.0 if nb == 6 else 6.0, nb)
        w = catalogs.uniform_weights(max(n, 1), seed=500 + k)[:n] if k % 2 else None
        npoint = 4 if k in (2, 4) else 3
        reqs.append((X, box_u, edges, npoint, None if npoint == 4 else w))
    return reqs


def single(gs, X, box_u, edges, npoint, w):
    g = gs.gs_build_graph(X, box_u, edges)
    if npoint == 4:
        e, o = gs.gs_count_4pcf_parity(g)
        return e, o, None
    if w is None:
        return gs.gs_count_3pcf(g), None, None
    c, ws = gs.gs_count_3pcf(g, w)
    return c, None, ws


@pytest.mark.parametrize("budget", [0, 8 << 20])
def test_server_mix_equals_single(gs, budget):
    reqs = make_requests()
    ref = [single(gs, *r) for r in reqs]
    with gs.gs_server(device_budget_bytes=budget, max_batch=3) as srv:
        tickets = [srv.submit(X, b, e, npoint=p, w=w) for X, b, e, p, w in reqs]
        for t, (rc, ro, rw), r in zip(tickets, ref, reqs):
            c, o, ws, info = srv.wait(t, timeout_s=120)
            assert np.array_equal(c, rc)
            if ro is not None:
                assert np.array_equal(o, ro)
            if rw is not None:
                assert np.array_equal(ws, rw)
            assert info["t_submit"] <= info["t_start"] <= info["t_done"]
    # one request is pinned to the oracle as well
    X, b, e, p, w = reqs[1]
    rc, rw = oracle.Graph(X, b, e).count_3pcf(w)
    assert np.array_equal(ref[1][0], rc)
    assert np.array_equal(ref[1][2], rw)


def test_server_rejects_bad_request(gs):
    with gs.gs_server() as srv:
        with pytest.raises(gs.GSError):
            srv.submit(np.zeros((3, 3), np.int32), 1000, [0, 10], npoint=5)
