"""CPU oracle for the binned 3pCF / 4pCF counts (test infrastructure only).

A plain, slow, obviously correct CPU implementation of the paper's
definitions (graph of Sec. 2.1, enumeration of Sec. 2.2, merge-walk of
Sec. 3.1, three-way walk of Eq. threeway, parity of Sec. 3.2 / Eq. volume,
disconnected term of Sec. 3.3 / Eq. disc, and the mu-binned 3pCF named in the
conclusions, in the reading stated at ``or_count_3pcf_mu``). It lives in
``gs_oracle.cpp`` and is loaded here with ctypes.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package. The CUDA library never uses it, and
it shares no code with the CUDA library: only the seeded input generators in
``catalogs`` serve both.

Every parity claim of the GPU path rests on this module, so its functions
are pinned by independent checks in ``tests/test_oracle_*.py``: brute force
over all tuples on tiny inputs, networkx clique enumeration, the Burnside
orbit counts, the Poisson closed form, mirror and rotation invariances and
the paper's parity injection test.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "_build", "libgs_oracle.so")
# A prebuilt oracle library to load instead (the planted-mistake tests
# point this at deliberately broken copies to show that the pins catch them).
_LIB_OVERRIDE = os.environ.get("GS_ORACLE_LIB")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (no GPU involved)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or \
            os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-pthread",
               "-ffp-contract=off", "-o", tmp, _SRC]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if _LIB_OVERRIDE:
        lib = ctypes.CDLL(_LIB_OVERRIDE)
    else:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    i64 = ctypes.c_int64
    ci = ctypes.c_int
    lib.or_quantize.argtypes = [P, i64, i64, ci, P]
    lib.or_quantize.restype = ci
    lib.or_graph_build.argtypes = [P, i64, i64, P, ci, ci, ci]
    lib.or_graph_build.restype = P
    lib.or_graph_num_edges.argtypes = [P]
    lib.or_graph_num_edges.restype = i64
    lib.or_graph_export.argtypes = [P, P, P, P]
    lib.or_graph_export.restype = None
    lib.or_graph_free.argtypes = [P]
    lib.or_graph_free.restype = None
    lib.or_num_configs.argtypes = [ci, ci]
    lib.or_num_configs.restype = i64
    lib.or_config_bins.argtypes = [ci, ci, i64, P, P]
    lib.or_config_bins.restype = ci
    lib.or_count_3pcf.argtypes = [P, P, P, P, i64, i64, ci]
    lib.or_count_3pcf.restype = ci
    lib.or_count_3pcf_mu.argtypes = [P, P, ci, P, P, ci]
    lib.or_count_3pcf_mu.restype = ci
    lib.or_count_4pcf.argtypes = [P, P, P, P, P, P, ci]
    lib.or_count_4pcf.restype = ci
    lib.or_pairs.argtypes = [P, P, P, P]
    lib.or_pairs.restype = ci
    lib.or_disconnected.argtypes = [P, P, P, P, P, P]
    lib.or_disconnected.restype = ci
    lib.or_connected_4pcf.argtypes = [P, P, P, P, P, P, P, P, P, ci]
    lib.or_connected_4pcf.restype = ci
    lib.or_count_4pcf_pix.argtypes = [P, P, P, P, P, P, ci]
    lib.or_count_4pcf_pix.restype = ci
    lib.or_direction_pixels.argtypes = [P, i64, P]
    lib.or_direction_pixels.restype = None
    lib.or_pixel_volumes.argtypes = [P, i64, P]
    lib.or_pixel_volumes.restype = None
    lib.or_exact_to_double.argtypes = [P, ci]
    lib.or_exact_to_double.restype = ctypes.c_double
    _lib = lib
    return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def quantize(pos, box_u: int, periodic: bool) -> np.ndarray:
    """Float positions (h^-1 Mpc) -> int32 lattice coordinates (N, 3)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    out = np.empty(pos.shape, dtype=np.int32)
    st = _load().or_quantize(_ptr(pos), pos.shape[0], int(box_u), int(bool(periodic)), _ptr(out))
    if st != 0:
        raise ValueError("coordinate outside the open box")
    return out


def exact_to_double(value: int, scale: int) -> float:
    """The oracle's final rounding step: the integer ``value`` (two's
    complement, |value| < 2^255) times 2^-scale, rounded to the nearest
    double with ties to even, as every exact weighted sum is rounded."""
    v = int(value)
    if not -(1 << 255) <= v < (1 << 255):
        raise ValueError("value outside the 256-bit accumulator")
    u = v & ((1 << 256) - 1)
    words = np.array([(u >> (64 * k)) & ((1 << 64) - 1) for k in range(4)], dtype=np.uint64)
    return float(_load().or_exact_to_double(_ptr(words), int(scale)))


def direction_pixels(d) -> np.ndarray:
    """Pixel (0..255) of integer direction vectors d [n][3]: 16 equal-width
    bands in z = cos(theta) times 16 equal sectors in phi, decided exactly."""
    d = np.ascontiguousarray(d, dtype=np.int64).reshape(-1, 3)
    out = np.empty(d.shape[0], dtype=np.uint8)
    _load().or_direction_pixels(_ptr(d), d.shape[0], _ptr(out))
    return out


def pixel_volumes(p) -> np.ndarray:
    """(u1 x u2) . u3 of the pixel centres of pixel triples p [n][3] (FP64)."""
    p = np.ascontiguousarray(p, dtype=np.int32).reshape(-1, 3)
    out = np.empty(p.shape[0], dtype=np.float64)
    _load().or_pixel_volumes(_ptr(p), p.shape[0], _ptr(out))
    return out


def num_configs(npoint: int, nb: int) -> int:
    return int(_load().or_num_configs(int(npoint), int(nb)))


def config_bins(npoint: int, nb: int, idx: int):
    bins = np.zeros(6, dtype=np.uint8)
    chiral = ctypes.c_int(0)
    st = _load().or_config_bins(int(npoint), int(nb), int(idx), _ptr(bins), ctypes.byref(chiral))
    if st != 0:
        raise IndexError(idx)
    return tuple(int(b) for b in bins[:npoint * (npoint - 1) // 2]), bool(chiral.value)


class Graph:
    """Full sorted adjacency (both directions) in the caller's labels."""

    def __init__(self, xyz, box_u: int, edges_u, method: str = "grid", nthreads: int | None = None):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.int32)
        self.n = self.xyz.shape[0]
        self.box_u = int(box_u)
        self.edges_u = np.ascontiguousarray(edges_u, dtype=np.int64)
        self.nb = len(self.edges_u) - 1
        self.nthreads = nthreads or default_threads()
        m = {"brute": 0, "grid": 1}[method]
        self._h = _load().or_graph_build(_ptr(self.xyz), self.n, self.box_u, _ptr(self.edges_u),
                                         self.nb, m, self.nthreads)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_graph_free(h)
            self._h = None

    def export(self):
        """(ptr int64[N+1], nbr int32[E], bin uint8[E]) with sorted rows."""
        e = _load().or_graph_num_edges(self._h)
        ptr = np.empty(self.n + 1, dtype=np.int64)
        nbr = np.empty(e, dtype=np.int32)
        b = np.empty(e, dtype=np.uint8)
        _load().or_graph_export(self._h, _ptr(ptr), _ptr(nbr), _ptr(b))
        return ptr, nbr, b

    def count_3pcf(self, w=None, hub_lo: int = 0, hub_hi: int = -1):
        nc = num_configs(3, self.nb)
        counts = np.zeros(nc, dtype=np.uint64)
        wsum = np.zeros(nc, dtype=np.float64) if w is not None else None
        wa = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
        st = _load().or_count_3pcf(self._h, _ptr(wa), _ptr(counts), _ptr(wsum), int(hub_lo),
                                   int(hub_hi), self.nthreads)
        if st != 0:
            raise ValueError(f"oracle 3pCF failed ({st})")
        return (counts, wsum) if w is not None else counts

    def count_3pcf_mu(self, nmu: int, w=None):
        """Anisotropic 3pCF: counts (and, with weights, exact weighted sums)
        of shape [C(nb+2,3), nmu + 1] by configuration and mu bin of the
        triangle's normal against the z axis; bin nmu holds the collinear
        triangles."""
        nc = num_configs(3, self.nb)
        counts = np.zeros((nc, nmu + 1), dtype=np.uint64)
        wsum = np.zeros((nc, nmu + 1), dtype=np.float64) if w is not None else None
        wa = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
        st = _load().or_count_3pcf_mu(self._h, _ptr(wa), int(nmu), _ptr(counts), _ptr(wsum),
                                      self.nthreads)
        if st != 0:
            raise ValueError(f"oracle mu-binned 3pCF failed ({st})")
        return (counts, wsum) if w is not None else counts

    def count_4pcf(self, w=None, pixel: bool = False):
        """Returns (even u64, odd i64) or, with weights, (even, odd, weven, wodd).
        pixel=True: odd channel from pixelised spoke directions (see
        direction_pixels), degenerate tetrahedra (|V| < 1e-9) excluded."""
        nc = num_configs(4, self.nb)
        even = np.zeros(nc, dtype=np.uint64)
        odd = np.zeros(nc, dtype=np.int64)
        we = np.zeros(nc, dtype=np.float64) if w is not None else None
        wo = np.zeros(nc, dtype=np.float64) if w is not None else None
        wa = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
        fn = _load().or_count_4pcf_pix if pixel else _load().or_count_4pcf
        st = fn(self._h, _ptr(wa), _ptr(even), _ptr(odd), _ptr(we), _ptr(wo), self.nthreads)
        if st != 0:
            raise ValueError(f"oracle 4pCF failed ({st})")
        return (even, odd, we, wo) if w is not None else (even, odd)

    def pairs(self, w=None):
        p = np.zeros(self.nb, dtype=np.uint64)
        wp = np.zeros(self.nb, dtype=np.float64)
        wa = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
        st = _load().or_pairs(self._h, _ptr(wa), _ptr(p), _ptr(wp))
        if st != 0:
            raise ValueError("oracle pairs failed")
        return (p, wp) if w is not None else p

    def disconnected(self, w=None, rr=None):
        """(pairs u64[nb], xi f64[nb], zeta_disc f64[n_orbits])."""
        no = num_configs(4, self.nb)
        p = np.zeros(self.nb, dtype=np.uint64)
        xi = np.zeros(self.nb, dtype=np.float64)
        z = np.zeros(no, dtype=np.float64)
        wa = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
        rra = None if rr is None else np.ascontiguousarray(rr, dtype=np.float64)
        st = _load().or_disconnected(self._h, _ptr(wa), _ptr(rra), _ptr(p), _ptr(xi), _ptr(z))
        if st != 0:
            raise ValueError(f"oracle disconnected failed ({st})")
        return p, xi, z


def connected_4pcf(g_dr: Graph, w_signed, g_r: Graph, w_r):
    """Signed-weight connected 4pCF (Sec. 3.3): dict of xi, zeta_even,
    zeta_odd, zeta_disc, zeta_conn."""
    nb = g_dr.nb
    nc = num_configs(4, nb)
    out = {k: np.zeros(nb if k == "xi" else nc) for k in
           ("xi", "zeta_even", "zeta_odd", "zeta_disc", "zeta_conn")}
    ws = np.ascontiguousarray(w_signed, dtype=np.float32)
    wr = np.ascontiguousarray(w_r, dtype=np.float32)
    st = _load().or_connected_4pcf(g_dr._h, _ptr(ws), g_r._h, _ptr(wr), _ptr(out["xi"]),
                                   _ptr(out["zeta_even"]), _ptr(out["zeta_odd"]),
                                   _ptr(out["zeta_disc"]), _ptr(out["zeta_conn"]), g_dr.nthreads)
    if st != 0:
        raise ValueError(f"oracle connected 4pCF failed ({st})")
    return out


# ----------------------------------------------------------------------------
# Configuration tooling (post-processing of the binned counts)

def _det_exact(M):
    """Determinant by the Leibniz sum over permutations, in exact arithmetic
    (ints or Fractions): fine for the 5 x 5 Cayley-Menger matrix."""
    import itertools
    n = len(M)
    total = 0
    for p in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if p[i] > p[j])
        t = -1 if inv & 1 else 1
        for i in range(n):
            t = t * M[i][p[i]]
        total += t
    return total


_SLOTS = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))


def cayley_menger_det(d2):
    """Cayley-Menger determinant of four points from their six squared
    distances in slot order (01, 02, 03, 12, 13, 23): the 5 x 5 matrix with
    a zero corner, a border of ones and the squared distances. It equals
    288 V^2 for a tetrahedron of volume V, and is not positive when the six
    lengths cannot be realised in three dimensions (Sec. 5.2, Cayley-Menger
    criterion)."""
    D = [[0] * 4 for _ in range(4)]
    for (i, j), x in zip(_SLOTS, d2):
        D[i][j] = D[j][i] = x
    M = [[0, 1, 1, 1, 1]] + [[1] + D[i] for i in range(4)]
    return _det_exact(M)


def config_mask_cm(nb: int, edges_u):
    """uint8 [n_orbits]: 1 when the orbit's six bin centres (midpoints of the
    bin edges, exact rationals) give a positive Cayley-Menger determinant."""
    from fractions import Fraction
    e = [int(x) for x in edges_u]
    centre = [Fraction(e[b] + e[b + 1], 2) for b in range(nb)]
    no = num_configs(4, nb)
    mask = np.zeros(no, dtype=np.uint8)
    for o in range(no):
        bins, _ = config_bins(4, nb, o)
        mask[o] = 1 if cayley_menger_det([centre[b] ** 2 for b in bins]) > 0 else 0
    return mask


def _perm_parity(p):
    return sum(1 for i in range(len(p)) for j in range(i + 1, len(p)) if p[i] > p[j]) & 1


def _relabel(t, p):
    """Tuple in slot order after vertex v takes the label p[v]."""
    d = {}
    for (i, j), x in zip(_SLOTS, t):
        a, b = sorted((p[i], p[j]))
        d[(a, b)] = x
    return tuple(d[s] for s in _SLOTS)


def _orbit_index(nb: int):
    """Every labelling of every orbit representative -> (orbit, parity of
    the relabelling, or None when both parities reach it)."""
    import itertools
    out = {}
    for o in range(num_configs(4, nb)):
        rep, _ = config_bins(4, nb, o)
        seen = {}
        for p in itertools.permutations(range(4)):
            t = _relabel(rep, p)
            par = _perm_parity(p)
            if t in seen and seen[t] != par:
                seen[t] = None
            elif t not in seen:
                seen[t] = par
        for t, par in seen.items():
            out[t] = (o, par)
    return out


def rebin_3pcf(nb_fine: int, nb_coarse: int, bin_map, counts, wsum=None):
    """Fine 3pCF counts -> coarse: each fine configuration's bins go through
    bin_map (fine bin -> coarse bin, or -1 to drop the configuration), are
    sorted and ranked among the coarse configurations (Sec. 5.1 combines
    caps after rebinning fine bins exactly). Weighted sums add in ascending
    fine index."""
    idx = {config_bins(3, nb_coarse, c)[0]: c for c in range(num_configs(3, nb_coarse))}
    out = np.zeros(num_configs(3, nb_coarse), dtype=np.uint64)
    wout = None if wsum is None else np.zeros(len(out), dtype=np.float64)
    for f in range(num_configs(3, nb_fine)):
        bins, _ = config_bins(3, nb_fine, f)
        m = [int(bin_map[b]) for b in bins]
        if min(m) < 0:
            continue
        c = idx[tuple(sorted(m))]
        out[c] += np.uint64(counts[f])
        if wout is not None:
            wout[c] = wout[c] + float(wsum[f])
    return out if wout is None else (out, wout)


def rebin_4pcf(nb_fine: int, nb_coarse: int, bin_map, even, odd=None, weven=None, wodd=None):
    """Fine 4pCF orbits -> coarse orbits. The fine representative's bins go
    through bin_map (a -1 drops it) in the fine representative's vertex
    labelling; the coarse orbit holding that labelled tuple is found, and
    odd counts change sign when the relabelling onto the coarse
    representative is an odd permutation (Sec. 3.2: the handedness of V
    follows the vertex order). Coarse orbits that are not chiral keep no odd
    part. Sums add in ascending fine index."""
    index = _orbit_index(nb_coarse)
    nc = num_configs(4, nb_coarse)
    chiral = [config_bins(4, nb_coarse, c)[1] for c in range(nc)]
    e_out = np.zeros(nc, dtype=np.uint64)
    o_out = np.zeros(nc, dtype=np.int64)
    we_out = np.zeros(nc) if weven is not None else None
    wo_out = np.zeros(nc) if wodd is not None else None
    for f in range(num_configs(4, nb_fine)):
        bins, _ = config_bins(4, nb_fine, f)
        m = tuple(int(bin_map[b]) for b in bins)
        if min(m) < 0:
            continue
        c, par = index[m]
        e_out[c] += np.uint64(even[f])
        if we_out is not None:
            we_out[c] = we_out[c] + float(weven[f])
        if not chiral[c]:
            continue
        s = -1 if par else 1
        if odd is not None:
            o_out[c] += s * int(odd[f])
        if wo_out is not None:
            wo_out[c] = wo_out[c] + s * float(wodd[f])
    return e_out, o_out, we_out, wo_out


def equilateral_3pcf(g: Graph, w=None):
    """Equilateral 3pCF read as the configurations (b, b, b): triangles with
    all three sides in bin b (the paper names the kernel without defining
    it). Counts uint64 [nb] (and weighted sums f64 [nb] with w), taken from
    the full 3pCF."""
    r = g.count_3pcf(w)
    c, ws = (r if w is not None else (r, None))
    idx = {config_bins(3, g.nb, k)[0]: k for k in range(num_configs(3, g.nb))}
    sel = [idx[(b, b, b)] for b in range(g.nb)]
    return (c[sel], ws[sel]) if w is not None else c[sel]
