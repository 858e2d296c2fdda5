"""Writes the oracle's results on the full-size workloads the bench times.

These cases take the CPU oracle minutes to tens of minutes, so their outputs
are computed once by this script and stored beside it; the GPU parity tests
(tests/test_gpu_fullsize.py) compare the CUDA path with them bin by bin. The
script calls only ``oracle`` (the CPU restatement of the paper's
definitions) and ``catalogs`` (the seeded generators); nothing here comes
from the CUDA path.

Each file records a SHA-256 of the lattice coordinates (and weights) it was
made from, so a test can tell that it regenerated the same catalogue.

Cases:
  rrr   3e6 uniform randoms, periodic L = 1000, rmax 40 in 20 bins, FP32
        weights U(0.5, 1.5): 3pCF counts and exact weighted sums (the
        dominant launch of the bench step).
  c3    2e5 Neyman-Scott points, periodic L = 400, rmax 30 in 8 bins:
        4pCF even and odd counts (pairs, xi and zeta_disc are cheap and are
        computed by the test itself).
  c4sub the 1e6-point sigma = 5 Neyman-Scott catalogue of the open L = 1494
        box, rmax 150 in 15 bins, cut to the sub-box [522, 972)^3 h^-1 Mpc
        (points kept in catalogue order): 3pCF counts and pair counts.

Usage: python tests/golden/make_fullsize.py [rrr] [c3] [c4sub]
"""
from __future__ import annotations

import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import catalogs  # noqa: E402
import oracle  # noqa: E402

# sub-box of the open-box workload, in h^-1 Mpc
C4_SUB_LO, C4_SUB_HI = 522.0, 972.0


def sha(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def inputs(case: str):
    """The case's lattice coordinates, box, edges and weights (or None)."""
    if case == "rrr":
        s = catalogs.WORKLOADS["ns1M_L1000_r40_nb20"]
        box_u = int(round(s["box"] * catalogs.LATTICE_PER_MPC))
        pos = catalogs.uniform(s["randoms"], s["box"], seed=s["random_seed"])
        w = catalogs.uniform_weights(s["randoms"], seed=s["weight_seed"] + 7)
        X = oracle.quantize(pos, box_u, True)
        return X, box_u, catalogs.bin_edges_u(s["rmin"], s["rmax"], s["nb"]), w
    if case == "c3":
        s = catalogs.draw("ns200k_L400_r30_nb8")
        return oracle.quantize(s["pos"], s["box_u"], True), s["box_u"], s["edges_u"], None
    if case == "c4sub":
        s = catalogs.draw("ns1M_open_L1494_r150_nb15")
        X = oracle.quantize(s["pos"], s["box_u"], False)
        lo = int(C4_SUB_LO * catalogs.LATTICE_PER_MPC)
        hi = int(C4_SUB_HI * catalogs.LATTICE_PER_MPC)
        keep = np.all((X >= lo) & (X < hi), axis=1)
        return np.ascontiguousarray(X[keep]), 0, s["edges_u"], None
    raise ValueError(case)


def make(case: str) -> str:
    t0 = time.time()
    X, box_u, edges, w = inputs(case)
    g = oracle.Graph(X, box_u, edges)
    out = {"n": np.int64(X.shape[0]), "box_u": np.int64(box_u), "edges_u": edges,
           "xyz_sha256": np.array(sha(X)), "w_sha256": np.array(sha(w) if w is not None else "")}
    if case == "rrr":
        out["counts"], out["wsum"] = g.count_3pcf(w)
    elif case == "c3":
        out["even"], out["odd"] = g.count_4pcf()
    else:
        out["counts"] = g.count_3pcf()
        out["pairs"] = g.pairs()
    out["oracle_seconds"] = np.float64(time.time() - t0)
    out["oracle_threads"] = np.int64(g.nthreads)
    path = os.path.join(HERE, f"fullsize_{case}.npz")
    np.savez_compressed(path, **out)
    return path


if __name__ == "__main__":
    for c in sys.argv[1:] or ["rrr", "c3", "c4sub"]:
        p = make(c)
        d = np.load(p)
        print(c, p, f"{float(d['oracle_seconds']):.0f} s", flush=True)
