"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Unweighted counts, pair counts and lattice coordinates must match bit for
bit. Weighted sums must match bit for bit too: both sides sum exactly (as
integers) and round the exact total once, to nearest with ties to even, by
two independent conversions. xi and zeta_disc are compared within 1e-12
relative: the two sides evaluate the analytic random pair counts RR with
FP64 operations in different orders.
"""
import json
import math
import os

import numpy as np
import pytest

import catalogs
import oracle

pytestmark = pytest.mark.gpu

RTOL = 1e-12
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


def rand_lattice(n, box_u, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, box_u, size=(n, 3)).astype(np.int32)


def clump(n, centre, spread, box_u, seed):
    rng = np.random.default_rng(seed)
    X = np.asarray(centre) + rng.integers(-spread, spread + 1, size=(n, 3))
    return np.mod(X, box_u).astype(np.int32)


def edge_set_from_gpu(gs, g):
    ptr, deg, nbr, b, perm = gs.gs_graph_export(g)
    rows = np.repeat(np.arange(len(deg)), deg)
    cols = np.concatenate([nbr[ptr[i]:ptr[i] + deg[i]] for i in range(len(deg))]) \
        if len(deg) else np.zeros(0, np.int64)
    bins = np.concatenate([b[ptr[i]:ptr[i] + deg[i]] for i in range(len(deg))]) \
        if len(deg) else np.zeros(0, np.uint8)
    a, c = perm[rows].astype(np.int64), perm[cols].astype(np.int64)
    lo, hi = np.minimum(a, c), np.maximum(a, c)
    key = (lo << 40) | (hi << 8) | bins.astype(np.int64)
    return np.sort(key), deg, ptr, nbr


def edge_set_from_oracle(og):
    ptr, nbr, b = og.export()
    rows = np.repeat(np.arange(og.n), np.diff(ptr))
    keep = nbr > rows
    key = (rows[keep].astype(np.int64) << 40) | (nbr[keep].astype(np.int64) << 8) | \
        b[keep].astype(np.int64)
    return np.sort(key)


# ----------------------------------------------------------------------------
# a1 quantisation


def test_quantize_bit_exact(gs, torch_mod):
    rng = np.random.default_rng(1)
    L = 250.0
    box_u = int(L * 1024)
    pos = rng.uniform(-L, 2 * L, size=(100_000, 3))
    pos[:10] = [[0.0, 0.0, 0.0], [L, L, L], [-1e-12, 1e-12, L - 1e-9], [1 / 1024, 2 / 1024, 3 / 1024],
                [L / 2, -L / 2, 1.5 * L], [-0.0, 0.5, 0.25], [1e-300, 7.0, 9.0],
                [249.99999999999997, 0.1, 0.2], [-250.0, -500.0, 500.0], [3.0, 3.0, 3.0]]
    ref = oracle.quantize(pos, box_u, True)
    assert np.array_equal(gs.gs_quantize(pos, box_u, True), ref)
    got = gs.gs_quantize(dev(torch_mod, pos), box_u, True)
    assert np.array_equal(got.cpu().numpy(), ref)
    inside = rng.uniform(0, L, size=(1000, 3))
    assert np.array_equal(gs.gs_quantize(inside, box_u, False), oracle.quantize(inside, box_u, False))
    with pytest.raises(gs.GSError) as e:
        gs.gs_quantize(pos, box_u, False)
    assert e.value.status == -2


# ----------------------------------------------------------------------------
# a2 graph


def adversarial(box_u, edges_u):
    pts = [[100, 100, 100], [100, 100, 100], [0, 0, 0], [box_u // 2, 0, 0],
           [box_u - 1, box_u - 1, box_u - 1]]
    base = np.array([box_u // 3, box_u // 5, box_u // 7])
    for e in edges_u:
        pts.append((base + [int(e), 0, 0]).tolist())
        pts.append((base + [0, int(e) - 1, 0]).tolist())
        pts.append((base + [0, 0, int(e) + 1]).tolist())
    return np.mod(np.array(pts, dtype=np.int64), box_u).astype(np.int32)


@pytest.mark.parametrize("periodic", [True, False])
def test_graph_edges_bit_exact(gs, periodic):
    box_u = 120_000
    edges = np.array([0, 2000, 3500, 5000, 6500, 8000], dtype=np.int64)
    X = np.concatenate([rand_lattice(20_000, box_u, 3), clump(3000, [50_000] * 3, 6000, box_u, 4),
                        adversarial(box_u, edges)])
    bu = box_u if periodic else 0
    g = gs.gs_build_graph(X, bu, edges)
    got, deg, ptr, nbr = edge_set_from_gpu(gs, g)
    og = oracle.Graph(X, bu, edges)
    ref = edge_set_from_oracle(og)
    assert np.array_equal(got, ref)
    # rows sorted ascending, only ids above the hub, padding to 16 bytes
    assert np.all(ptr % 4 == 0)
    for i in range(0, len(deg), 97):
        r = nbr[ptr[i]:ptr[i] + deg[i]]
        assert np.all(np.diff(r) > 0) and (len(r) == 0 or r[0] > i)
    info = gs.gs_graph_info(g)
    assert info["edges"] == len(ref) and info["max_degree"] == deg.max()
    # variant 1: the 64-bit candidate test (the default here is the 32-bit one)
    g64 = gs.gs_build_graph(X, bu, edges, variant=1)
    assert np.array_equal(edge_set_from_gpu(gs, g64)[0], ref)


@pytest.mark.parametrize("periodic", [True, False])
def test_graph_dense_cells_and_wide_bins(gs, periodic):
    """A clump whose cell stencil holds more points than the row pass stages
    in shared memory (4,096: those cells read their points from global
    memory), and E_nb above 2^16 (the 64-bit candidate test)."""
    rng = np.random.default_rng(17)
    box_u = 400_000
    X = np.concatenate([rng.integers(0, box_u, size=(6000, 3)),
                        200_000 + rng.integers(-2000, 2001, size=(6000, 3))]).astype(np.int32)
    bu = box_u if periodic else 0
    for edges in (np.array([0, 1000, 3000, 6000], dtype=np.int64),
                  np.array([0, 30_000, 70_000, 90_000], dtype=np.int64)):
        g = gs.gs_build_graph(X, bu, edges)
        got = edge_set_from_gpu(gs, g)[0]
        assert np.array_equal(got, edge_set_from_oracle(oracle.Graph(X, bu, edges)))


# ----------------------------------------------------------------------------
# a3 triangles


def run3(gs, torch, X, box_u, edges, w=None):
    g = gs.gs_build_graph(dev(torch, X), box_u, edges)
    if w is None:
        return gs.gs_count_3pcf(g, like=dev(torch, np.zeros(1))).cpu().numpy()
    c, ws = gs.gs_count_3pcf(g, dev(torch, w))
    return c.cpu().numpy(), ws.cpu().numpy()


def test_3pcf_uniform20k_full_size(gs, torch_mod):
    """20,000 uniform points, L=200, rmax 20 in 10 bins: every bin bit-exact."""
    s = catalogs.draw("uniform20k_L200_r20_nb10")
    X = oracle.quantize(s["pos"], s["box_u"], True)
    og = oracle.Graph(X, s["box_u"], s["edges_u"])
    ref = og.count_3pcf()
    got = run3(gs, torch_mod, X, s["box_u"], s["edges_u"])
    assert ref.sum() > 10_000_000
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("periodic,seed", [(True, 11), (False, 12)])
def test_3pcf_clustered_weighted(gs, torch_mod, periodic, seed):
    L = 150.0
    box_u = int(L * 1024)
    pos = catalogs.neyman_scott(30_000, L, seed=seed, sigma=2.0, periodic=periodic)
    w = catalogs.uniform_weights(pos.shape[0], seed=seed + 1)
    X = oracle.quantize(pos, box_u, periodic)
    edges = catalogs.bin_edges_u(0.0, 12.0, 8)
    bu = box_u if periodic else 0
    og = oracle.Graph(X, bu, edges)
    rc, rw = og.count_3pcf(w)
    gc, gw = run3(gs, torch_mod, X, bu, edges, w)
    assert np.array_equal(gc, rc)
    assert np.array_equal(gw, rw)
    # unweighted call on the same graph agrees with the weighted call's counts
    assert np.array_equal(run3(gs, torch_mod, X, bu, edges), rc)
    # every kernel gives the same answer: the default pair kernel (0, and 4
    # with computed configuration ranks) and the merge-walk kernel (512 and
    # every bit of its own paths: hash path in 64-word segments (1), hub rows
    # from global memory (2), a 2 KB table (8), compaction (32), the prefetch
    # ring (64))
    g = gs.gs_build_graph(X, bu, edges)
    ex_c, ex_w = gs.gs_count_3pcf(g, w)
    assert np.array_equal(ex_c, rc)
    assert np.array_equal(ex_w, rw)
    for variant in (4, 512, 516, 1, 2, 6, 8, 10, 32, 34, 36, 40, 64, 68, 72, 96):
        vc, vw = gs.gs_count_3pcf(g, w, variant=variant)
        assert np.array_equal(vc, rc), variant
        assert np.array_equal(vw, rw), variant
        # exact sums are identical bit for bit whichever path found them
        assert np.array_equal(gs.gs_count_3pcf(g, w, variant=variant)[1], ex_w)


def test_3pcf_signed_weights(gs, torch_mod):
    """Weights of both signs take the general carry chain of the exact sums
    (nonnegative weights take a cheaper one): every launch path agrees with
    the oracle's exact sums, and negating every weight negates the sums."""
    L = 150.0
    box_u = int(L * 1024)
    pos = catalogs.neyman_scott(30_000, L, seed=15, sigma=2.0, periodic=True)
    X = oracle.quantize(pos, box_u, True)
    w = catalogs.uniform_weights(len(X), seed=16)
    sign = np.where(np.random.default_rng(17).random(len(X)) < 0.5, -1.0, 1.0)
    w = (w * sign).astype(np.float32)
    edges = catalogs.bin_edges_u(0.0, 12.0, 8)
    rc, rw = oracle.Graph(X, box_u, edges).count_3pcf(w)
    assert np.any(rw < 0) and np.any(rw > 0)
    g = gs.gs_build_graph(X, box_u, edges)
    for variant in (0, 4, 512, 1, 32, 64):
        gc, gw = gs.gs_count_3pcf(g, w, variant=variant)
        assert np.array_equal(gc, rc), variant
        assert np.array_equal(gw, rw), variant
    _, gn = gs.gs_count_3pcf(g, -w)
    assert np.array_equal(gn, -gs.gs_count_3pcf(g, w)[1])


def test_weighted_sum_rounds_to_nearest_at_a_tie(gs, torch_mod):
    """One triangle (and one tetrahedron) whose weight product
    (1 + 2^-23)^2 (1 + 2^-7 + 2^-23) has its bits at 2^0, -7, -22, -23, -29,
    -45, -46, -53 and -69: the first dropped bit (2^-53) is set and a bit 16
    places further down decides the rounding, so a conversion that kept only
    the top 64 bits would see an exact tie and round down. The correctly
    rounded sum rounds up; both sides must give exactly Fraction's value."""
    from fractions import Fraction
    a = np.float32(1 + 2.0 ** -23)
    b = np.float32(1 + 2.0 ** -7 + 2.0 ** -23)
    exact = Fraction(float(a)) ** 2 * Fraction(float(b))
    truncated = float(Fraction(int(exact * 2 ** 63), 2 ** 63))
    assert float(exact) != truncated
    box_u = 100_000
    edges = np.array([0, 100, 200], dtype=np.int64)
    X = np.array([[500, 500, 500], [550, 500, 500], [500, 550, 500], [500, 500, 550]],
                 dtype=np.int32)
    for sign in (1.0, -1.0):
        w3 = np.array([a, a, sign * b], dtype=np.float32)
        c, ws = gs.gs_count_3pcf(gs.gs_build_graph(X[:3], box_u, edges), w3)
        rc, rw = oracle.Graph(X[:3], box_u, edges).count_3pcf(w3)
        assert c.sum() == 1 and np.array_equal(c, rc)
        assert ws[c.argmax()] == sign * float(exact) and np.array_equal(ws, rw)
        w4 = np.array([a, a, sign * b, 1.0], dtype=np.float32)
        g4 = gs.gs_build_graph(X, box_u, edges)
        e, o, we, wo = gs.gs_count_4pcf_parity(g4, w4)
        re, ro, rwe, rwo = oracle.Graph(X, box_u, edges).count_4pcf(w4)
        assert e.sum() == 1 and np.array_equal(e, re) and np.array_equal(o, ro)
        assert we[e.argmax()] == sign * float(exact)
        assert np.array_equal(we, rwe) and np.array_equal(wo, rwo)


@pytest.mark.parametrize("rmin,rmax,nb", [(0.0, 12.0, 8), (1.0, 9.0, 8), (0.0, 10.3, 7)])
def test_3pcf_pair_kernel_binning_modes(gs, torch_mod, rmin, rmax, nb):
    """The pair kernel bins a pair's squared distance three ways, chosen by
    the bin edges: linear bins from zero (E_b = b m 2^t) by a square root,
    edges whose squares share a power-of-two factor (here E_b = 1024 (b + 1),
    with r_min > 0) by one table lookup that also rejects pairs closer than
    E_0, and any other edges by a range test and a comparison. Each against
    the oracle and the merge-walk kernel, weighted and unweighted."""
    L = 100.0
    box_u = int(L * 1024)
    pos = catalogs.neyman_scott(15_000, L, seed=int(10 * rmax) + nb, sigma=1.5)
    X = oracle.quantize(pos, box_u, True)
    w = catalogs.uniform_weights(len(X), seed=nb)
    edges = catalogs.bin_edges_u(rmin, rmax, nb)
    rc, rw = oracle.Graph(X, box_u, edges).count_3pcf(w)
    assert rc.sum() > 100_000
    g = gs.gs_build_graph(X, box_u, edges)
    for variant in (0, 4, 512):
        c, ws = gs.gs_count_3pcf(g, w, variant=variant)
        assert np.array_equal(c, rc) and np.array_equal(ws, rw), variant
        assert np.array_equal(gs.gs_count_3pcf(g, variant=variant), rc), variant


def wide_weights(n, seed, span_log2=20):
    """FP32 weights whose magnitudes span 2^span_log2 (log-uniform), both signs."""
    rng = np.random.default_rng(seed)
    mag = np.exp2(rng.uniform(-span_log2 / 2, span_log2 / 2, size=n)) * rng.uniform(0.5, 1.5, n)
    return (mag * np.where(rng.random(n) < 0.3, -1.0, 1.0)).astype(np.float32)


@pytest.mark.parametrize("periodic", [True, False])
def test_3pcf_wide_weights(gs, torch_mod, periodic):
    """Weights spanning 2^20 take the split-weight path (exact sums of the
    products of A + t B at four points t, interpolated and rounded once):
    bit for bit the oracle's exact sums, on both triangle kernels."""
    L = 120.0
    box_u = int(L * 1024)
    pos = catalogs.neyman_scott(20_000, L, seed=171, sigma=2.0, periodic=periodic)
    X = oracle.quantize(pos, box_u, periodic)
    w = wide_weights(len(X), seed=172)
    assert np.abs(w).max() / np.abs(w).min() > 2 ** 19
    edges = catalogs.bin_edges_u(0.0, 12.0, 8)
    bu = box_u if periodic else 0
    rc, rw = oracle.Graph(X, bu, edges).count_3pcf(w)
    g = gs.gs_build_graph(X, bu, edges)
    for variant in (0, 512):
        gc, gw = gs.gs_count_3pcf(g, w, variant=variant)
        assert np.array_equal(gc, rc) and np.array_equal(gw, rw), variant
    gc, gw = gs.gs_count_3pcf(g, dev(torch_mod, w))
    assert np.array_equal(gw.cpu().numpy(), rw)


def test_4pcf_wide_weights(gs, torch_mod):
    box_u = 80_000
    rng = np.random.default_rng(181)
    X = np.concatenate([rng.integers(0, box_u, size=(4000, 3)),
                        np.mod(40_000 + rng.integers(-5000, 5001, size=(300, 3)), box_u)])
    X = X.astype(np.int32)
    w = wide_weights(X.shape[0], seed=182)
    edges = np.array([0, 2500, 5000, 7000], dtype=np.int64)
    og = oracle.Graph(X, box_u, edges)
    re, ro, rwe, rwo = og.count_4pcf(w)
    ge, go, gwe, gwo = run4(gs, torch_mod, X, box_u, edges, w)
    assert np.array_equal(ge, re) and np.array_equal(go, ro)
    assert np.array_equal(gwe, rwe) and np.array_equal(gwo, rwo)
    pe, po, pwe, pwo = og.count_4pcf(w, pixel=True)
    g = gs.gs_build_graph(X, box_u, edges)
    qe, qo, qwe, qwo = gs.gs_count_4pcf_parity_pix(g, w)
    assert np.array_equal(qe, pe) and np.array_equal(qo, po)
    assert np.array_equal(qwe, pwe) and np.array_equal(qwo, pwo)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 5])
def test_3pcf_tiny_and_empty(gs, torch_mod, n):
    box_u = 100_000
    edges = np.array([0, 5000, 10000], dtype=np.int64)
    X = clump(n, [500, 500, 500], 3000, box_u, n) if n else np.zeros((0, 3), np.int32)
    ref = oracle.Graph(X, box_u, edges).count_3pcf()
    assert np.array_equal(run3(gs, torch_mod, X, box_u, edges), ref)


def test_3pcf_coincident_points(gs, torch_mod):
    """50 points on one lattice site: C(50,3) triangles in configuration (0,0,0)."""
    X = np.full((50, 3), 777, dtype=np.int32)
    edges = np.array([0, 100, 200], dtype=np.int64)
    got = run3(gs, torch_mod, X, 100_000, edges)
    assert got[0] == math.comb(50, 3) and got.sum() == got[0]


@pytest.mark.parametrize("periodic", [True, False])
def test_3pcf_long_rows_segmented(gs, torch_mod, periodic):
    """variant 1 stages hub rows in 64-word segments, so rows of ~70-200
    neighbours run through the multi-segment path (binary-searched spoke
    starts, spokes read from global memory)."""
    L = 120.0
    box_u = int(L * 1024)
    pos = catalogs.neyman_scott(20_000, L, seed=24, sigma=2.0, periodic=periodic)
    X = oracle.quantize(pos, box_u, periodic)
    edges = catalogs.bin_edges_u(0.0, 14.0, 7)
    bu = box_u if periodic else 0
    w = catalogs.uniform_weights(X.shape[0], seed=23)
    og = oracle.Graph(X, bu, edges)
    ptr, _, _ = og.export()
    assert np.diff(ptr).max() > 2 * 64
    rc, rw = og.count_3pcf(w)
    g = gs.gs_build_graph(dev(torch_mod, X), bu, edges)
    gc, gw = gs.gs_count_3pcf(g, dev(torch_mod, w), variant=1)
    assert np.array_equal(gc.cpu().numpy(), rc)
    assert np.array_equal(gw.cpu().numpy(), rw)
    _, gx = gs.gs_count_3pcf(g, dev(torch_mod, w), variant=1)
    assert np.array_equal(gx.cpu().numpy(), rw)


def test_3pcf_host_and_device_pointers(gs, torch_mod):
    box_u = 60_000
    X = rand_lattice(5000, box_u, 31)
    edges = np.array([0, 3000, 6000], dtype=np.int64)
    ref = oracle.Graph(X, box_u, edges).count_3pcf()
    g_host = gs.gs_build_graph(X, box_u, edges)
    assert np.array_equal(gs.gs_count_3pcf(g_host), ref)  # host in, host out
    out = torch_mod.zeros(len(ref), dtype=torch_mod.uint64, device="cuda")
    gs.gs_count_3pcf(g_host, counts=out)  # device out
    assert np.array_equal(out.cpu().numpy(), ref)


# ----------------------------------------------------------------------------
# a4 / a5 tetrahedra and parity


def run4(gs, torch, X, box_u, edges, w=None):
    g = gs.gs_build_graph(dev(torch, X), box_u, edges)
    like = dev(torch, np.zeros(1))
    if w is None:
        e, o = gs.gs_count_4pcf_parity(g, like=like)
        c = gs.gs_count_4pcf(g, like=like)
        assert np.array_equal(c.cpu().numpy(), e.cpu().numpy())
        return e.cpu().numpy(), o.cpu().numpy()
    e, o, we, wo = gs.gs_count_4pcf_parity(g, dev(torch, w))
    return e.cpu().numpy(), o.cpu().numpy(), we.cpu().numpy(), wo.cpu().numpy()


@pytest.mark.parametrize("periodic,nb,seed", [(True, 4, 41), (False, 6, 42), (True, 8, 43)])
def test_4pcf_parity_clustered(gs, torch_mod, periodic, nb, seed):
    L = 100.0
    box_u = int(L * 1024)
    pos = catalogs.neyman_scott(12_000, L, seed=seed, sigma=1.5, periodic=periodic)
    X = oracle.quantize(pos, box_u, periodic)
    edges = catalogs.bin_edges_u(0.0, 9.0, nb)
    bu = box_u if periodic else 0
    og = oracle.Graph(X, bu, edges)
    re, ro = og.count_4pcf()
    ge, go = run4(gs, torch_mod, X, bu, edges)
    assert re.sum() > 100_000 and np.abs(ro).sum() > 0
    assert np.array_equal(ge, re)
    assert np.array_equal(go, ro)
    # variant 4 bins the three non-hub edges by binary search over the edges
    # instead of the squared-distance buckets
    g = gs.gs_build_graph(dev(torch_mod, X), bu, edges)
    be, bo = gs.gs_count_4pcf_parity(g, like=dev(torch_mod, np.zeros(1)), variant=4)
    assert np.array_equal(be.cpu().numpy(), re) and np.array_equal(bo.cpu().numpy(), ro)
    # variant 8: 64 orbits in shared memory, the others counted in global memory
    he, ho = gs.gs_count_4pcf_parity(g, like=dev(torch_mod, np.zeros(1)), variant=8)
    assert np.array_equal(he.cpu().numpy(), re) and np.array_equal(ho.cpu().numpy(), ro)


def test_4pcf_weighted(gs, torch_mod):
    box_u = 80_000
    X = np.concatenate([rand_lattice(4000, box_u, 51), clump(300, [40_000] * 3, 5000, box_u, 52)])
    w = catalogs.uniform_weights(X.shape[0], seed=53)
    edges = np.array([0, 2500, 5000, 7000], dtype=np.int64)
    og = oracle.Graph(X, box_u, edges)
    re, ro, rwe, rwo = og.count_4pcf(w)
    ge, go, gwe, gwo = run4(gs, torch_mod, X, box_u, edges, w)
    assert np.array_equal(ge, re) and np.array_equal(go, ro)
    assert np.array_equal(gwe, rwe) and np.array_equal(gwo, rwo)


@pytest.fixture(scope="module")
def many_orbits():
    """8 bins (12,496 orbits, more than the weighted kernel keeps in shared
    memory): clustered points with signed weights, and the oracle's sums."""
    L = 100.0
    box_u = int(L * 1024)
    pos = catalogs.neyman_scott(12_000, L, seed=71, sigma=1.5, periodic=True)
    X = oracle.quantize(pos, box_u, True)
    rng = np.random.default_rng(72)
    w = (catalogs.uniform_weights(len(X), seed=73) *
         np.where(rng.random(len(X)) < 0.4, -1.0, 1.0)).astype(np.float32)
    edges = catalogs.bin_edges_u(0.0, 9.0, 8)
    og = oracle.Graph(X, box_u, edges)
    return X, box_u, edges, w, og.count_4pcf(w), og.count_4pcf(w, pixel=True)


@pytest.mark.parametrize("variant,windows", [(0, 0), (8, 0), (1, 0), (0, 3), (8, 3)])
def test_4pcf_weighted_many_orbits(gs, torch_mod, many_orbits, variant, windows):
    """Weighted sums with more orbits than shared slots: the orbits met most
    often in a sample of hubs keep per-hub sums in shared memory, the rest go
    to the global sums directly (variant 8 keeps only 64 slots, variant 1
    sends every hub to the global path; windows > 0 samples the first row
    window only)."""
    X, box_u, edges, w, ref, _ = many_orbits
    assert np.count_nonzero(ref[0]) > 1000 and np.abs(ref[1]).sum() > 0
    g = gs.gs_build_graph(dev(torch_mod, X), box_u, edges, force_windows=windows)
    got = gs.gs_count_4pcf_parity(g, dev(torch_mod, w), variant=variant)
    for a, b in zip(got, ref):
        assert np.array_equal(a.cpu().numpy(), b)


def test_4pcf_ten_bins(gs, torch_mod):
    """nb = 10 (45,475 orbits): more orbits than shared memory holds beside
    the hub workspace, so both the unweighted and the weighted kernels keep
    some orbits (the most frequent in a sample of hubs, or the first ones
    where the sampling kernel does not fit) in shared memory and send the
    others to the global counts and sums."""
    L = 60.0
    box_u = int(L * 1024)
    pos = catalogs.neyman_scott(3000, L, seed=81, sigma=1.5, periodic=True)
    X = oracle.quantize(pos, box_u, True)
    w = catalogs.uniform_weights(len(X), seed=82)
    edges = catalogs.bin_edges_u(0.0, 7.0, 10)
    ref = oracle.Graph(X, box_u, edges).count_4pcf(w)
    assert ref[0].sum() > 10_000
    g = gs.gs_build_graph(dev(torch_mod, X), box_u, edges)
    got = gs.gs_count_4pcf_parity(g, dev(torch_mod, w))
    for a, b in zip(got, ref):
        assert np.array_equal(a.cpu().numpy(), b)
    like = dev(torch_mod, np.zeros(1))
    e, o = gs.gs_count_4pcf_parity(g, like=like)
    assert np.array_equal(e.cpu().numpy(), ref[0]) and np.array_equal(o.cpu().numpy(), ref[1])
    assert np.array_equal(gs.gs_count_4pcf(g, like=like).cpu().numpy(), ref[0])


@pytest.mark.parametrize("variant", [0, 8])
def test_4pcf_pixel_weighted_many_orbits(gs, torch_mod, many_orbits, variant):
    X, box_u, edges, w, _, ref = many_orbits
    g = gs.gs_build_graph(dev(torch_mod, X), box_u, edges)
    got = gs.gs_count_4pcf_parity_pix(g, dev(torch_mod, w), variant=variant)
    for a, b in zip(got, ref):
        assert np.array_equal(a.cpu().numpy(), b)


@pytest.mark.parametrize("periodic", [True, False])
def test_4pcf_global_workspace(gs, torch_mod, periodic):
    """variant 1 runs every hub in the launch whose workspace lives in global
    memory (the path taken by rows longer than the shared-memory capacity)."""
    L = 100.0
    box_u = int(L * 1024)
    pos = catalogs.neyman_scott(12_000, L, seed=63, sigma=1.5, periodic=periodic)
    X = oracle.quantize(pos, box_u, periodic)
    edges = catalogs.bin_edges_u(0.0, 9.0, 5)
    bu = box_u if periodic else 0
    og = oracle.Graph(X, bu, edges)
    re, ro = og.count_4pcf()
    g = gs.gs_build_graph(dev(torch_mod, X), bu, edges)
    ge, go = gs.gs_count_4pcf_parity(g, like=dev(torch_mod, np.zeros(1)), variant=1)
    assert np.array_equal(ge.cpu().numpy(), re) and np.array_equal(go.cpu().numpy(), ro)


@pytest.mark.parametrize("mirrored_fraction", [0.0, 0.3, 0.5])
def test_parity_injection_gpu(gs, torch_mod, mirrored_fraction):
    """Sec. 4.9 injection test: odd = N_L - N_R exactly at the injected orbit."""
    gold = json.load(open(os.path.join(GOLDEN, "injection_tetrahedron.json")))
    edges = np.array(gold["edges_u"], dtype=np.int64)
    n = gold["n_struct"]
    _, lat, mirrored = catalogs.lattice_tetrahedra(np.array(gold["shape_u"]), n, mirrored_fraction,
                                                   gold["box_u"], int(edges[-1]) + 1, seed=78)
    ge, go = run4(gs, torch_mod, lat.astype(np.int32), gold["box_u"], edges)
    nb = len(edges) - 1
    k = [gs.gs_config_bins(4, nb, i)[0] for i in range(gs.gs_num_configs(4, nb))].index(tuple(gold["rep"]))
    assert ge[k] == n and ge.sum() == n
    assert go[k] == gold["left_sign"] * (int((~mirrored).sum()) - int(mirrored.sum()))


# ----------------------------------------------------------------------------
# a6 pairs, xi, zeta_disc


@pytest.mark.parametrize("weighted", [False, True])
def test_disconnected_parity(gs, torch_mod, weighted):
    L = 120.0
    box_u = int(L * 1024)
    pos = catalogs.neyman_scott(25_000, L, seed=71, sigma=2.0)
    X = oracle.quantize(pos, box_u, True)
    w = catalogs.uniform_weights(X.shape[0], seed=72) if weighted else None
    edges = catalogs.bin_edges_u(0.0, 10.0, 6)
    og = oracle.Graph(X, box_u, edges)
    rp, rxi, rz = og.disconnected(w)
    g = gs.gs_build_graph(dev(torch_mod, X), box_u, edges)
    p, xi, z = gs.gs_disconnected_4pcf(g, None if w is None else dev(torch_mod, w),
                                       like=dev(torch_mod, np.zeros(1)))
    assert np.array_equal(p.cpu().numpy(), rp)
    np.testing.assert_allclose(xi.cpu().numpy(), rxi, rtol=RTOL, atol=RTOL)
    np.testing.assert_allclose(z.cpu().numpy(), rz, rtol=RTOL, atol=RTOL)
    # caller-supplied RR, open box
    rr = np.linspace(1e4, 2e4, 6)
    og2 = oracle.Graph(X, 0, edges)
    rp2, rxi2, rz2 = og2.disconnected(w, rr=rr)
    g2 = gs.gs_build_graph(X, 0, edges)
    p2, xi2, z2 = gs.gs_disconnected_4pcf(g2, w, rr=rr)
    assert np.array_equal(p2, rp2)
    np.testing.assert_allclose(xi2, rxi2, rtol=RTOL, atol=RTOL)
    np.testing.assert_allclose(z2, rz2, rtol=RTOL, atol=RTOL)


def connected_case(periodic, seed):
    """Clustered data and uniform randoms (twice as many) in one box, with
    data weights normalised to +1 and random weights to -1 (Sec. 3.3)."""
    L = 110.0
    box_u = int(L * 1024)
    D = oracle.quantize(catalogs.neyman_scott(4000, L, seed=seed, sigma=1.5, periodic=periodic),
                        box_u, periodic)
    R = oracle.quantize(catalogs.uniform(8000, L, seed=seed + 1), box_u, periodic)
    wd = catalogs.uniform_weights(len(D), seed=seed + 2).astype(np.float64)
    wr = catalogs.uniform_weights(len(R), seed=seed + 3).astype(np.float64)
    w_signed = np.concatenate([wd / wd.sum(), -wr / wr.sum()]).astype(np.float32)
    w_r = (wr / wr.sum()).astype(np.float32)
    U = np.concatenate([D, R])
    edges = catalogs.bin_edges_u(0.0, 11.0, 4)
    return U, R, (box_u if periodic else 0), edges, w_signed, w_r


def assert_estimator_close(got, want):
    """Both sides round exact sums once; every later step is one IEEE op, so
    the results agree to a few ulps of the operands' scale (conn subtracts
    two nearly equal terms, hence the scale |even| + |disc|)."""
    for k in ("xi", "zeta_even", "zeta_odd", "zeta_disc"):
        a, b = np.asarray(got[k]), want[k]
        assert np.array_equal(np.isnan(a), np.isnan(b)), k
        m = ~np.isnan(b)
        np.testing.assert_allclose(a[m], b[m], rtol=RTOL, atol=0, err_msg=k)
    scale = np.abs(want["zeta_even"]) + np.abs(want["zeta_disc"])
    a, b = np.asarray(got["zeta_conn"]), want["zeta_conn"]
    assert np.array_equal(np.isnan(a), np.isnan(b)), "zeta_conn"
    # an empty RRRR bin gives the same infinity on both sides
    m = ~np.isnan(b) & (a != b)
    assert np.all(np.abs(a[m] - b[m]) <= RTOL * scale[m])


@pytest.mark.parametrize("periodic,seed", [(True, 91), (False, 93)])
def test_connected_4pcf_signed_estimator(gs, torch_mod, periodic, seed):
    U, R, bu, edges, w_signed, w_r = connected_case(periodic, seed)
    want = oracle.connected_4pcf(oracle.Graph(U, bu, edges), w_signed,
                                 oracle.Graph(R, bu, edges), w_r)
    assert np.isfinite(want["zeta_even"]).sum() > 20
    assert np.nansum(np.abs(want["zeta_odd"])) > 0  # empty RRRR bins give NaN
    # host arrays in, host arrays out
    got = gs.gs_connected_4pcf(gs.gs_build_graph(U, bu, edges), w_signed,
                               gs.gs_build_graph(R, bu, edges), w_r)
    assert_estimator_close(got, want)
    # device arrays, and an out-of-core union graph (three windows)
    gd = gs.gs_build_graph(dev(torch_mod, U), bu, edges, force_windows=3)
    got_d = gs.gs_connected_4pcf(gd, dev(torch_mod, w_signed),
                                 gs.gs_build_graph(dev(torch_mod, R), bu, edges),
                                 dev(torch_mod, w_r))
    for k in got:
        assert got_d[k].is_cuda
        assert np.array_equal(got_d[k].cpu().numpy(), got[k], equal_nan=True), k


def test_connected_4pcf_errors(gs, torch_mod):
    U, R, bu, edges, w_signed, w_r = connected_case(True, 95)
    gd = gs.gs_build_graph(U[:2000], bu, edges)
    e_other = edges.copy()
    e_other[-1] -= 1
    gr_other = gs.gs_build_graph(R[:1000], bu, e_other)
    with pytest.raises(gs.GSError) as e:
        gs.gs_connected_4pcf(gd, w_signed[:2000], gr_other, w_r[:1000])
    assert e.value.status == -1
    gr = gs.gs_build_graph(R[:1000], bu, edges)
    with pytest.raises(gs.GSError) as e:
        gs.gs_connected_4pcf(gd, w_signed[:2000], gr, w_r[:1000], shards=2)
    assert e.value.status == -1
    wide = w_signed[:2000].copy()
    wide[0] = 1e6  # magnitudes beyond the exact fixed-point range
    with pytest.raises(gs.GSError) as e:
        gs.gs_connected_4pcf(gd, wide, gr, w_r[:1000])
    assert e.value.status == -6
    out = gs.gs_connected_4pcf(gd, w_signed[:2000], gr, w_r[:1000])
    assert out["xi"].shape == (len(edges) - 1,)


# ----------------------------------------------------------------------------
# Full-size workloads


@pytest.fixture(scope="module")
def ns1m(gs):
    s = catalogs.draw("ns1M_L1000_r40_nb20")
    X = oracle.quantize(s["pos"], s["box_u"], True)
    w = catalogs.uniform_weights(X.shape[0], seed=s["weight_seed"])
    return s, X, w


def test_full_size_ddd_bit_exact(gs, torch_mod, ns1m):
    """1e6 Neyman-Scott points, L=1000, rmax 40 in 20 bins: DDD against the
    oracle on every bin, unweighted bit-exact and weighted to 1e-12."""
    s, X, w = ns1m
    og = oracle.Graph(X, s["box_u"], s["edges_u"])
    rc, rw = og.count_3pcf(w)
    gc, gw = run3(gs, torch_mod, X, s["box_u"], s["edges_u"], w)
    assert rc.sum() > 1e9
    assert np.array_equal(gc, rc)
    assert np.array_equal(gw, rw)
    g = gs.gs_build_graph(dev(torch_mod, X), s["box_u"], s["edges_u"])
    _, gx = gs.gs_count_3pcf(g, dev(torch_mod, w))
    assert np.array_equal(gx.cpu().numpy(), rw)


def test_full_size_rrr_properties(gs, torch_mod):
    """3e6 uniform randoms, L=1000, rmax 40 in 20 bins (too large for the
    oracle): mirror and relabelling invariance hold bit for bit, the
    triangle total matches the Poisson closed form C(N,3) p^2 15/32, and the
    exact weighted sums obey the same invariances and exact scalings."""
    s = catalogs.draw("ns1M_L1000_r40_nb20")
    N = s["randoms"]
    pos = catalogs.uniform(N, s["box"], seed=s["random_seed"])
    box_u = s["box_u"]
    X = oracle.quantize(pos, box_u, True)
    c0 = run3(gs, torch_mod, X, box_u, s["edges_u"])
    Xm = X.copy()
    Xm[:, 0] = np.mod(-Xm[:, 0].astype(np.int64), box_u).astype(np.int32)
    assert np.array_equal(run3(gs, torch_mod, Xm, box_u, s["edges_u"]), c0)
    perm = np.random.default_rng(9).permutation(N)
    assert np.array_equal(run3(gs, torch_mod, X[perm], box_u, s["edges_u"]), c0)
    p = 4 * math.pi * float(s["edges_u"][-1]) ** 3 / 3 / float(box_u) ** 3
    expect = math.comb(N, 3) * p * p * 15 / 32
    sd = math.sqrt(expect) * 30  # generous: triangle counts are strongly correlated
    assert abs(float(c0.sum()) - expect) < 5 * sd
    # the launch configuration the bench times: counts with exact weighted sums.
    # Exact sums are invariant bit for bit under the mirror and a relabelling,
    # equal the counts for unit weights and scale by exactly 8 when every
    # weight doubles (2w is exact in FP32).
    w = catalogs.uniform_weights(N, seed=s["weight_seed"] + 7)
    cw, ws = run3(gs, torch_mod, X, box_u, s["edges_u"], w)
    assert np.array_equal(cw, c0)
    assert np.array_equal(run3(gs, torch_mod, Xm, box_u, s["edges_u"], w)[1], ws)
    assert np.array_equal(run3(gs, torch_mod, X[perm], box_u, s["edges_u"], w[perm])[1], ws)
    ones = np.ones(N, dtype=np.float32)
    assert np.array_equal(run3(gs, torch_mod, X, box_u, s["edges_u"], ones)[1],
                          c0.astype(np.float64))
    assert np.array_equal(run3(gs, torch_mod, X, box_u, s["edges_u"], 2 * w)[1], 8 * ws)


def test_4pcf_parity_clustered_workload_density(gs, torch_mod):
    """Neyman-Scott points at the density of the 2e5-point L=400 workload
    (2.5e4 points, L=200; mean degree about 360), rmax 30 in 8 bins: every
    even and odd bin against the oracle (the full 2e5 catalogue takes the
    oracle many minutes)."""
    L = 200.0
    box_u = int(L * 1024)
    pos = catalogs.neyman_scott(25_000, L, seed=4, sigma=2.0)
    X = oracle.quantize(pos, box_u, True)
    edges = catalogs.bin_edges_u(0.0, 30.0, 8)
    og = oracle.Graph(X, box_u, edges)
    re, ro = og.count_4pcf()
    ge, go = run4(gs, torch_mod, X, box_u, edges)
    assert re.sum() > 1e9
    assert np.array_equal(ge, re) and np.array_equal(go, ro)


def test_full_size_out_of_core_workload(gs, torch_mod):
    """1e6 Neyman-Scott points (sigma 5) in an open box L=1494, rmax 150 in 15
    bins (about 1.2e12 triangles, too many for the oracle): a graph streamed
    in forced windows counts exactly what the resident graph counts, and the
    mirror image x -> L-1-x counts the same."""
    s = catalogs.draw("ns1M_open_L1494_r150_nb15")
    box_u, edges = s["box_u"], s["edges_u"]
    X = oracle.quantize(s["pos"], box_u, False)
    Xd = dev(torch_mod, X)
    c0 = gs.gs_count_3pcf(gs.gs_build_graph(Xd, 0, edges), like=Xd).cpu().numpy()
    assert c0.sum() > 1e12
    g3 = gs.gs_build_graph(Xd, 0, edges, force_windows=3)
    assert gs.gs_graph_info(g3)["windows"] >= 3
    assert np.array_equal(gs.gs_count_3pcf(g3, like=Xd).cpu().numpy(), c0)
    del g3
    Xm = X.copy()
    Xm[:, 0] = (box_u - 1 - Xm[:, 0].astype(np.int64)).astype(np.int32)
    Xmd = dev(torch_mod, Xm)
    cm = gs.gs_count_3pcf(gs.gs_build_graph(Xmd, 0, edges), like=Xmd).cpu().numpy()
    assert np.array_equal(cm, c0)


def test_expired_wait_reports_timeout_and_context_survives(gs, torch_mod):
    """A bounded device wait that runs out (variant 16 gives the first
    staging wait no polls) makes the call return GS_ETIMEOUT without a
    fault; the next calls on the same graph and device succeed."""
    box_u = 60_000
    X = rand_lattice(8000, box_u, 81)
    edges = np.array([0, 3000, 6000], dtype=np.int64)
    g = gs.gs_build_graph(X, box_u, edges)
    ref = gs.gs_count_3pcf(g)
    for _ in range(2):
        with pytest.raises(gs.GSError) as e:
            gs.gs_count_3pcf(g, variant=16)
        assert e.value.status == -5
        assert np.array_equal(gs.gs_count_3pcf(g), ref)
    torch_mod.cuda.synchronize()
    assert np.array_equal(oracle.Graph(X, box_u, edges).count_3pcf(), ref)
