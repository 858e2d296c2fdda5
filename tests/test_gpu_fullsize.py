"""Full-size parity on the workloads the bench times, bin by bin.

The oracle needs minutes to tens of minutes on these catalogues, so its
results were computed once by tests/golden/make_fullsize.py (which calls
only the oracle and the seeded generators) and stored as
tests/golden/fullsize_*.npz. Each test regenerates the same catalogue, checks
its SHA-256 against the stored one (if the host produced a different
catalogue, the oracle is run here instead of trusting the file) and compares
the CUDA path through the C ABI with the oracle's values:

* 3e6 uniform randoms, periodic L = 1000, rmax 40 in 20 bins, FP32 weights:
  counts and exact weighted sums, bit for bit, in the launch configuration
  the bench times (the dominant launch of its step).
* 2e5 Neyman-Scott points, periodic L = 400, rmax 30 in 8 bins: 4pCF even
  and odd channels bit for bit; pairs, xi and zeta_disc against the oracle
  run here (one sweep, cheap).
* The 1e6-point open-box rmax-150 catalogue cut to a 450 h^-1 Mpc sub-box:
  3pCF and pair counts bit for bit, resident and streamed through forced
  out-of-core windows.
"""
import hashlib
import os
import sys

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))
import make_fullsize  # noqa: E402


@pytest.fixture(scope="module")
def gs():
    import torch
    assert torch.cuda.is_available()
    import paper_2607_06604_gb300 as m
    return m


def sha(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def expected(case):
    """(inputs, stored oracle results), recomputing the results with the
    oracle when this host generated a different catalogue."""
    X, box_u, edges, w = make_fullsize.inputs(case)
    d = dict(np.load(os.path.join(HERE, "golden", f"fullsize_{case}.npz")))
    same = str(d["xyz_sha256"]) == sha(X) and \
        str(d["w_sha256"]) == (sha(w) if w is not None else "")
    if not same:
        path = make_fullsize.make(case)
        d = dict(np.load(path))
    assert np.array_equal(d["edges_u"], edges) and int(d["box_u"]) == box_u
    return (X, box_u, edges, w), d


def test_fullsize_randoms_3pcf_weighted(gs):
    import torch
    (X, box_u, edges, w), d = expected("rrr")
    Xd = torch.from_numpy(X).cuda()
    wd = torch.from_numpy(w).cuda()
    g = gs.gs_build_graph(Xd, box_u, edges)
    c, ws = gs.gs_count_3pcf(g, wd)
    c, ws = c.cpu().numpy(), ws.cpu().numpy()
    assert d["counts"].sum() > 1e11
    assert np.array_equal(c, d["counts"])
    assert np.array_equal(ws, d["wsum"])


def test_fullsize_4pcf_parity_and_disconnected(gs):
    import torch
    (X, box_u, edges, _), d = expected("c3")
    Xd = torch.from_numpy(X).cuda()
    g = gs.gs_build_graph(Xd, box_u, edges)
    e, o = gs.gs_count_4pcf_parity(g, like=Xd)
    assert d["even"].sum() > 5e10 and np.abs(d["odd"]).sum() > 0
    assert np.array_equal(e.cpu().numpy(), d["even"])
    assert np.array_equal(o.cpu().numpy(), d["odd"])
    p, xi, z = gs.gs_disconnected_4pcf(g, like=Xd)
    rp, rxi, rz = oracle.Graph(X, box_u, edges).disconnected()
    assert np.array_equal(p.cpu().numpy(), rp)
    np.testing.assert_allclose(xi.cpu().numpy(), rxi, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(z.cpu().numpy(), rz, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("windows", [0, 3])
def test_fullsize_open_box_subbox(gs, windows):
    import torch
    (X, box_u, edges, _), d = expected("c4sub")
    Xd = torch.from_numpy(X).cuda()
    g = gs.gs_build_graph(Xd, 0, edges, force_windows=windows)
    nw = gs.gs_graph_info(g)["windows"]
    assert nw == 1 if windows == 0 else nw >= 2
    c = gs.gs_count_3pcf(g, like=Xd).cpu().numpy()
    assert d["counts"].sum() > 1e9
    assert np.array_equal(c, d["counts"])
    p = gs.gs_disconnected_4pcf(g, rr=np.ones(len(edges) - 1), like=Xd, zeta=False)[0]
    assert np.array_equal(p.cpu().numpy(), d["pairs"])
