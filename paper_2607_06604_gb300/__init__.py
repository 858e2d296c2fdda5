"""Python binding of libgramsci_gb300 (GB300 / sm_103a query engine).

Binned 3pCF / 4pCF tuple counts over a fixed-radius neighbour graph after
GRAMSCI v2: graph of Sec. 2.1, hub-and-spoke enumeration of Sec. 2.2 /
Sec. 3.1, parity channels of Sec. 3.2, disconnected term of Sec. 3.3.

Every function below has the name of the C entry point it marshals
arguments for (include/gramsci_gb300.h); all arithmetic runs in the CUDA
library. Array arguments may be NumPy arrays (host) or torch tensors (host
or CUDA); outputs are allocated like the first array input unless given.
A missing or unbuildable library raises at import time: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = [
    "GSError", "Options", "GraphStats", "Graph", "gs_quantize", "gs_build_graph",
    "gs_graph_info", "gs_graph_tri_words", "gs_graph_export", "gs_count_3pcf", "gs_tune_3pcf", "gs_count_3pcf_noalloc", "gs_count_3pcf_batch", "gs_count_3pcf_equilateral", "gs_count_3pcf_mu", "gs_count_4pcf",
    "gs_count_4pcf_parity", "gs_count_4pcf_parity_pix", "gs_direction_pixels",
    "gs_disconnected_4pcf", "gs_connected_4pcf", "gs_config_mask_cm",
    "gs_rebin_3pcf", "gs_rebin_4pcf", "gs_num_configs", "gs_config_bins",
    "gs_free_graph", "gs_strerror", "gs_kernel_launches", "gs_server", "gs_plan", "lib_path",
]


class GSError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {gs_strerror(status)} ({status})")
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_uint64), ("force_windows", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("flags", ctypes.c_uint32), ("shard", ctypes.c_int32), ("shards", ctypes.c_int32),
                ("kernel_ms", ctypes.POINTER(ctypes.c_double))]


class GraphStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nb", ctypes.c_int32), ("max_degree", ctypes.c_int32),
                ("edges", ctypes.c_int64), ("edge_slots", ctypes.c_int64),
                ("probe_words", ctypes.c_int64), ("bytes_per_edge", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("windows", ctypes.c_int32),
                ("cells", ctypes.c_int32), ("walk_words", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerConfig(ctypes.Structure):
    _fields_ = [("device_budget_bytes", ctypes.c_uint64), ("max_batch", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("xyz", ctypes.c_void_p), ("n", ctypes.c_int64), ("box_u", ctypes.c_int64),
                ("edges_u", ctypes.c_void_p), ("nb", ctypes.c_int32), ("npoint", ctypes.c_int32),
                ("w", ctypes.c_void_p), ("counts", ctypes.c_void_p), ("odd", ctypes.c_void_p),
                ("wsum", ctypes.c_void_p)]


class TicketInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


def _load():
    # (re)build in-tree when missing or older than its sources; raises when
    # nvcc is missing or the build fails
    path = _build.build()
    lib = ctypes.CDLL(path)
    P, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    OP = ctypes.POINTER(Options)
    sig = {
        "gs_quantize": ([P, i64, i64, ci, P, OP], ci),
        "gs_build_graph": ([P, i64, i64, P, ci, OP, ctypes.POINTER(P)], ci),
        "gs_graph_info": ([P, ctypes.POINTER(GraphStats)], ci),
        "gs_graph_export": ([P, P, P, P, P, P], ci),
        "gs_graph_tri_words": ([P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)], ci),
        "gs_count_3pcf": ([P, P, P, P, OP], ci),
        "gs_count_4pcf": ([P, P, P, P, OP], ci),
        "gs_count_3pcf_batch": ([P, ctypes.c_int32, P, P, P, OP], ci),
        "gs_count_3pcf_noalloc": ([P, P, OP], ci),
        "gs_tune_3pcf": ([P, P, OP, ctypes.POINTER(ctypes.c_int32)], ci),
        "gs_plan_3pcf_batch": ([P, ctypes.c_int32, P, OP, ctypes.POINTER(P)], ci),
        "gs_plan_launch": ([P, P], ci),
        "gs_plan_wait": ([P, P], ci),
        "gs_plan_destroy": ([P], None),
        "gs_count_4pcf_parity": ([P, P, P, P, P, P, OP], ci),
        "gs_count_4pcf_parity_pix": ([P, P, P, P, P, P, OP], ci),
        "gs_direction_pixels": ([P, ctypes.c_int64, P, OP], ci),
        "gs_disconnected_4pcf": ([P, P, P, P, P, P, OP], ci),
        "gs_connected_4pcf": ([P, P, P, P, P, P, P, P, P, OP], ci),
        "gs_count_3pcf_equilateral": ([P, P, P, P, OP], ci),
        "gs_count_3pcf_mu": ([P, P, ci, P, P, OP], ci),
        "gs_config_mask_cm": ([ci, P, P, ctypes.POINTER(i64), OP], ci),
        "gs_rebin_3pcf": ([ci, ci, P, P, P, P, P, OP], ci),
        "gs_rebin_4pcf": ([ci, ci, P, P, P, P, P, P, P, P, P, OP], ci),
        "gs_num_configs": ([ci, ci, ctypes.POINTER(i64)], ci),
        "gs_config_bins": ([ci, ci, i64, P, ctypes.POINTER(ci)], ci),
        "gs_free_graph": ([P], None),
        "gs_strerror": ([ci], ctypes.c_char_p),
        "gs_kernel_launches": ([], ctypes.c_uint64),
        "gs_server_create": ([ctypes.POINTER(ServerConfig), ctypes.POINTER(P)], ci),
        "gs_server_submit": ([P, ctypes.POINTER(Request), ctypes.POINTER(i64)], ci),
        "gs_server_wait": ([P, i64, ctypes.c_double, ctypes.POINTER(TicketInfo)], ci),
        "gs_server_destroy": ([P], ci),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    return lib, path


_lib, lib_path = _load()


def gs_kernel_launches() -> int:
    return int(_lib.gs_kernel_launches())


def gs_strerror(status: int) -> str:
    return _lib.gs_strerror(int(status)).decode()


def _check(status: int, where: str):
    if status != 0:
        raise GSError(status, where)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return x.ctypes.data_as(ctypes.c_void_p)


def _empty_like_input(ref, shape, np_dtype):
    """Output on the same side (host NumPy / torch device) as ``ref``."""
    if ref is not None and _is_torch(ref):
        import torch
        tdt = {np.uint64: torch.uint64, np.int64: torch.int64, np.float64: torch.float64,
               np.int32: torch.int32, np.uint8: torch.uint8}[np_dtype]
        return torch.empty(shape, dtype=tdt, device=ref.device)
    return np.empty(shape, dtype=np_dtype)


def _options(stream=None, budget=0, force_windows=0, variant=0, kernel_ms=None, shard=0,
             shards=0):
    o = Options()
    o.shard = int(shard)
    o.shards = int(shards)
    if kernel_ms is not None:  # a ctypes.c_double receiving the kernel time
        o.kernel_ms = ctypes.pointer(kernel_ms)
    o.device_budget_bytes = int(budget)
    o.force_windows = int(force_windows)
    o.variant = int(variant)
    if stream is not None:
        o.stream = ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
    return o


def gs_num_configs(npoint: int, nb: int) -> int:
    n = ctypes.c_int64(0)
    _check(_lib.gs_num_configs(int(npoint), int(nb), ctypes.byref(n)), "gs_num_configs")
    return n.value


def gs_config_bins(npoint: int, nb: int, idx: int):
    bins = np.zeros(6, dtype=np.uint8)
    chiral = ctypes.c_int(0)
    _check(_lib.gs_config_bins(int(npoint), int(nb), int(idx), _ptr(bins), ctypes.byref(chiral)),
           "gs_config_bins")
    k = 3 if npoint == 3 else 6
    return tuple(int(b) for b in bins[:k]), bool(chiral.value)


def gs_quantize(pos, box_u: int, periodic: bool, out=None, **opts):
    """Float positions (h^-1 Mpc) -> int32 lattice coordinates."""
    n = int(pos.shape[0])
    if out is None:
        out = _empty_like_input(pos, (n, 3), np.int32)
    o = _options(**opts)
    _check(_lib.gs_quantize(_ptr(pos), n, int(box_u), int(bool(periodic)), _ptr(out),
                            ctypes.byref(o)), "gs_quantize")
    return out


class Graph:
    """Owning handle of a device-resident gs_graph."""

    def __init__(self, handle, nb: int, n: int):
        self._h = handle
        self.nb = nb
        self.n = n

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            _lib.gs_free_graph(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gs_build_graph(xyz, box_u: int, edges_u, **opts) -> Graph:
    n = int(xyz.shape[0])
    edges = np.ascontiguousarray(np.asarray(edges_u, dtype=np.int64))
    nb = len(edges) - 1
    h = ctypes.c_void_p()
    o = _options(**opts)
    _check(_lib.gs_build_graph(_ptr(xyz), n, int(box_u), _ptr(edges), nb, ctypes.byref(o),
                               ctypes.byref(h)), "gs_build_graph")
    return Graph(h, nb, n)


def gs_free_graph(g: Graph):
    g.close()


def gs_graph_info(g: Graph) -> dict:
    s = GraphStats()
    _check(_lib.gs_graph_info(g.handle, ctypes.byref(s)), "gs_graph_info")
    return s.as_dict()


def gs_graph_tri_words(g: Graph):
    """(triangles, sum over triangles i<j<k of |N+(k)|) of the graph."""
    t = ctypes.c_int64(0)
    w = ctypes.c_int64(0)
    _check(_lib.gs_graph_tri_words(g.handle, ctypes.byref(t), ctypes.byref(w)),
           "gs_graph_tri_words")
    return int(t.value), int(w.value)


def gs_graph_export(g: Graph):
    """Oriented CSR in internal labels: (ptr, deg, nbr, bin, perm) NumPy arrays."""
    info = gs_graph_info(g)
    n, slots = info["n"], info["edge_slots"]
    ptr = np.empty(n + 1, np.int64)
    deg = np.empty(n, np.int32)
    nbr = np.empty(slots, np.int32)
    b = np.empty(slots, np.uint8)
    perm = np.empty(n, np.int32)
    _check(_lib.gs_graph_export(g.handle, _ptr(ptr), _ptr(deg), _ptr(nbr), _ptr(b), _ptr(perm)),
           "gs_graph_export")
    return ptr, deg, nbr, b, perm


def gs_count_3pcf(g: Graph, w=None, counts=None, wsum=None, like=None, **opts):
    """Triangle counts per configuration (and exact weighted sums when w is given)."""
    nc = gs_num_configs(3, g.nb)
    ref = like if like is not None else w
    if counts is None:
        counts = _empty_like_input(ref, (nc,), np.uint64)
    if w is not None and wsum is None:
        wsum = _empty_like_input(ref, (nc,), np.float64)
    o = _options(**opts)
    _check(_lib.gs_count_3pcf(g.handle, _ptr(w), _ptr(counts), _ptr(wsum), ctypes.byref(o)),
           "gs_count_3pcf")
    return (counts, wsum) if w is not None else counts


def gs_tune_3pcf(g: Graph, w=None, **opts) -> int:
    """Time the 3pCF launch variants on a sample of g; variant=-1 then uses the best."""
    best = ctypes.c_int32(0)
    o = _options(**opts)
    _check(_lib.gs_tune_3pcf(g.handle, _ptr(w), ctypes.byref(o), ctypes.byref(best)),
           "gs_tune_3pcf")
    return int(best.value)


def gs_count_3pcf_noalloc(g: Graph, counts=None, like=None, **opts):
    """Unweighted triangle counts through the entry point that allocates no
    device memory (fixed scratch inside the library; see the C header)."""
    nc = gs_num_configs(3, g.nb)
    if counts is None:
        counts = _empty_like_input(like, (nc,), np.uint64)
    o = _options(**opts)
    _check(_lib.gs_count_3pcf_noalloc(g.handle, _ptr(counts), ctypes.byref(o)),
           "gs_count_3pcf_noalloc")
    return counts


def gs_count_3pcf_batch(graphs, ws=None, like=None, **opts):
    """One persistent launch over several graphs; returns [(counts, wsum|None)]."""
    n = len(graphs)
    nc = gs_num_configs(3, graphs[0].nb)
    ref = like if like is not None else (ws[0] if ws else None)
    counts = [_empty_like_input(ref, (nc,), np.uint64) for _ in graphs]
    wsums = [_empty_like_input(ref, (nc,), np.float64) for _ in graphs] if ws else None
    P = ctypes.c_void_p
    harr = (P * n)(*[g.handle for g in graphs])
    carr = (P * n)(*[_ptr(c) for c in counts])
    warr = (P * n)(*[_ptr(x) for x in ws]) if ws else None
    sarr = (P * n)(*[_ptr(x) for x in wsums]) if ws else None
    o = _options(**opts)
    _check(_lib.gs_count_3pcf_batch(harr, n, warr, carr, sarr, ctypes.byref(o)),
           "gs_count_3pcf_batch")
    return [(c, wsums[k] if ws else None) for k, c in enumerate(counts)]


def gs_count_4pcf(g: Graph, w=None, counts=None, wsum=None, like=None, **opts):
    nc = gs_num_configs(4, g.nb)
    ref = like if like is not None else w
    if counts is None:
        counts = _empty_like_input(ref, (nc,), np.uint64)
    if w is not None and wsum is None:
        wsum = _empty_like_input(ref, (nc,), np.float64)
    o = _options(**opts)
    _check(_lib.gs_count_4pcf(g.handle, _ptr(w), _ptr(counts), _ptr(wsum), ctypes.byref(o)),
           "gs_count_4pcf")
    return (counts, wsum) if w is not None else counts


def gs_count_4pcf_parity(g: Graph, w=None, like=None, pix=False, **opts):
    """(even u64, odd i64) or, with weights, (even, odd, weven, wodd).
    pix=True: the odd channel from pixelised spoke directions
    (gs_count_4pcf_parity_pix)."""
    nc = gs_num_configs(4, g.nb)
    ref = like if like is not None else w
    even = _empty_like_input(ref, (nc,), np.uint64)
    odd = _empty_like_input(ref, (nc,), np.int64)
    we = _empty_like_input(ref, (nc,), np.float64) if w is not None else None
    wo = _empty_like_input(ref, (nc,), np.float64) if w is not None else None
    o = _options(**opts)
    fn, name = ((_lib.gs_count_4pcf_parity_pix, "gs_count_4pcf_parity_pix") if pix else
                (_lib.gs_count_4pcf_parity, "gs_count_4pcf_parity"))
    _check(fn(g.handle, _ptr(w), _ptr(even), _ptr(odd), _ptr(we), _ptr(wo), ctypes.byref(o)), name)
    return (even, odd, we, wo) if w is not None else (even, odd)


def gs_count_4pcf_parity_pix(g: Graph, w=None, like=None, **opts):
    """Parity 4pCF with the odd channel from pixelised spoke directions."""
    return gs_count_4pcf_parity(g, w, like=like, pix=True, **opts)


def gs_direction_pixels(dirs, **opts):
    """Direction pixels (uint8) of integer vectors [n][3] (host or device)."""
    if not _is_torch(dirs):
        dirs = np.ascontiguousarray(dirs, dtype=np.int32)
    n = int(dirs.shape[0])
    out = _empty_like_input(dirs, (n,), np.uint8)
    o = _options(**opts)
    _check(_lib.gs_direction_pixels(_ptr(dirs), n, _ptr(out), ctypes.byref(o)),
           "gs_direction_pixels")
    return out


def gs_disconnected_4pcf(g: Graph, w=None, rr=None, like=None, zeta=True, **opts):
    """(pairs u64[nb], xi f64[nb], zeta_disc f64[n_orbits] or None)."""
    ref = like if like is not None else w
    pairs = _empty_like_input(ref, (g.nb,), np.uint64)
    xi = _empty_like_input(ref, (g.nb,), np.float64)
    z = _empty_like_input(ref, (gs_num_configs(4, g.nb),), np.float64) if zeta else None
    if rr is not None and not _is_torch(rr):
        rr = np.ascontiguousarray(rr, dtype=np.float64)
    o = _options(**opts)
    _check(_lib.gs_disconnected_4pcf(g.handle, _ptr(w), _ptr(rr), _ptr(pairs), _ptr(xi), _ptr(z),
                                     ctypes.byref(o)), "gs_disconnected_4pcf")
    return pairs, xi, z


def gs_connected_4pcf(g_dr: Graph, w_signed, g_r: Graph, w_r, **opts):
    """Signed-weight connected 4pCF: dict of xi [nb] and zeta_even, zeta_odd,
    zeta_disc, zeta_conn [n_orbits] (host NumPy, or torch tensors on the
    weights' device when the weights are torch tensors)."""
    if not _is_torch(w_signed):
        w_signed = np.ascontiguousarray(w_signed, dtype=np.float32)
    if not _is_torch(w_r):
        w_r = np.ascontiguousarray(w_r, dtype=np.float32)
    no = gs_num_configs(4, g_dr.nb)
    out = {"xi": _empty_like_input(w_signed, (g_dr.nb,), np.float64)}
    for k in ("zeta_even", "zeta_odd", "zeta_disc", "zeta_conn"):
        out[k] = _empty_like_input(w_signed, (no,), np.float64)
    o = _options(**opts)
    _check(_lib.gs_connected_4pcf(g_dr.handle, _ptr(w_signed), g_r.handle, _ptr(w_r),
                                  _ptr(out["xi"]), _ptr(out["zeta_even"]), _ptr(out["zeta_odd"]),
                                  _ptr(out["zeta_disc"]), _ptr(out["zeta_conn"]), ctypes.byref(o)),
           "gs_connected_4pcf")
    return out


def gs_count_3pcf_equilateral(g: Graph, w=None, like=None, **opts):
    """Triangles with all three sides in bin b, for each b (uint64 [nb]), and
    with w the exact weighted sums (float64 [nb])."""
    ref = like if like is not None else w
    counts = _empty_like_input(ref, (g.nb,), np.uint64)
    wsum = _empty_like_input(ref, (g.nb,), np.float64) if w is not None else None
    o = _options(**opts)
    _check(_lib.gs_count_3pcf_equilateral(g.handle, _ptr(w), _ptr(counts), _ptr(wsum),
                                          ctypes.byref(o)), "gs_count_3pcf_equilateral")
    return (counts, wsum) if w is not None else counts


def gs_count_3pcf_mu(g: Graph, nmu: int, w=None, like=None, **opts):
    """Anisotropic 3pCF: uint64 [n_conf, nmu + 1] counts by configuration and
    mu bin of the triangle's normal against the z axis (the last bin holds
    collinear triangles), and with w the exact weighted sums (float64, same
    shape)."""
    ref = like if like is not None else w
    shape = (gs_num_configs(3, g.nb), int(nmu) + 1)
    counts = _empty_like_input(ref, shape, np.uint64)
    wsum = _empty_like_input(ref, shape, np.float64) if w is not None else None
    o = _options(**opts)
    _check(_lib.gs_count_3pcf_mu(g.handle, _ptr(w), int(nmu), _ptr(counts), _ptr(wsum),
                                 ctypes.byref(o)), "gs_count_3pcf_mu")
    return (counts, wsum) if w is not None else counts


def gs_config_mask_cm(nb: int, edges_u, **opts):
    """(uint8 mask [n_orbits], number kept): orbits whose bin centres form a
    tetrahedron by the Cayley-Menger criterion."""
    edges = np.ascontiguousarray(edges_u, dtype=np.int64)
    mask = np.empty(gs_num_configs(4, nb), np.uint8)
    kept = ctypes.c_int64(0)
    o = _options(**opts)
    _check(_lib.gs_config_mask_cm(int(nb), _ptr(edges), _ptr(mask), ctypes.byref(kept),
                                  ctypes.byref(o)), "gs_config_mask_cm")
    return mask, int(kept.value)


def _rebin_in(x, dtype):
    return None if x is None else (x if _is_torch(x) else np.ascontiguousarray(x, dtype=dtype))


def gs_rebin_3pcf(nb_fine: int, nb_coarse: int, bin_map, counts=None, wsum=None, **opts):
    """Coarse (counts, wsum) from fine ones; either may be None."""
    bm = _rebin_in(bin_map, np.int32)
    counts, wsum = _rebin_in(counts, np.uint64), _rebin_in(wsum, np.float64)
    ref = counts if counts is not None else wsum
    nc = gs_num_configs(3, nb_coarse)
    oc = None if counts is None else _empty_like_input(ref, (nc,), np.uint64)
    ow = None if wsum is None else _empty_like_input(ref, (nc,), np.float64)
    o = _options(**opts)
    _check(_lib.gs_rebin_3pcf(int(nb_fine), int(nb_coarse), _ptr(bm), _ptr(counts), _ptr(wsum),
                              _ptr(oc), _ptr(ow), ctypes.byref(o)), "gs_rebin_3pcf")
    return oc, ow


def gs_rebin_4pcf(nb_fine: int, nb_coarse: int, bin_map, even=None, odd=None, weven=None,
                  wodd=None, **opts):
    """Coarse (even, odd, weven, wodd) from fine ones; any may be None."""
    bm = _rebin_in(bin_map, np.int32)
    ins = [_rebin_in(even, np.uint64), _rebin_in(odd, np.int64), _rebin_in(weven, np.float64),
           _rebin_in(wodd, np.float64)]
    ref = next((x for x in ins if x is not None), None)
    nc = gs_num_configs(4, nb_coarse)
    outs = [None if x is None else _empty_like_input(ref, (nc,), dt)
            for x, dt in zip(ins, (np.uint64, np.int64, np.float64, np.float64))]
    o = _options(**opts)
    _check(_lib.gs_rebin_4pcf(int(nb_fine), int(nb_coarse), _ptr(bm), *[_ptr(x) for x in ins],
                              *[_ptr(x) for x in outs], ctypes.byref(o)), "gs_rebin_4pcf")
    return tuple(outs)


class gs_server:
    """Request loop (gs_server_* in the C ABI). Submitted inputs are copied;
    output arrays are allocated here (host NumPy) and handed back by wait()."""

    def __init__(self, device_budget_bytes: int = 0, max_batch: int = 0):
        cfg = ServerConfig(int(device_budget_bytes), int(max_batch), 0)
        self._h = ctypes.c_void_p()
        _check(_lib.gs_server_create(ctypes.byref(cfg), ctypes.byref(self._h)), "gs_server_create")
        self._live = {}

    def submit(self, xyz, box_u, edges_u, npoint=3, w=None) -> int:
        xyz = np.ascontiguousarray(xyz, dtype=np.int32)
        edges = np.ascontiguousarray(edges_u, dtype=np.int64)
        nb = len(edges) - 1
        nc = gs_num_configs(npoint, nb)
        counts = np.zeros(nc, np.uint64)
        odd = np.zeros(nc, np.int64) if npoint == 4 else None
        wsum = np.zeros(nc, np.float64) if w is not None else None
        wa = None if w is None else np.ascontiguousarray(w, dtype=np.float32)
        r = Request(_ptr(xyz), xyz.shape[0], int(box_u), _ptr(edges), nb, npoint, _ptr(wa),
                    _ptr(counts), _ptr(odd), _ptr(wsum))
        t = ctypes.c_int64(0)
        _check(_lib.gs_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)), "gs_server_submit")
        self._live[t.value] = (counts, odd, wsum)
        return t.value

    def wait(self, ticket: int, timeout_s: float = -1.0):
        """(counts, odd|None, wsum|None, info dict)."""
        info = TicketInfo()
        st = _lib.gs_server_wait(self._h, int(ticket), float(timeout_s), ctypes.byref(info))
        _check(st, "gs_server_wait")
        counts, odd, wsum = self._live.pop(ticket)
        return counts, odd, wsum, {"t_submit": info.t_submit, "t_start": info.t_start,
                                   "t_done": info.t_done}

    def close(self):
        if self._h:
            _lib.gs_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class gs_plan:
    """A batched 3pCF count recorded once into a CUDA graph and replayed
    (gs_plan_* in the C ABI). Outputs are torch CUDA tensors kept here."""

    def __init__(self, graphs, **opts):
        import torch
        self._graphs = list(graphs)  # the plan refers to them
        nc = gs_num_configs(3, self._graphs[0].nb)
        self.counts = [torch.zeros(nc, dtype=torch.uint64, device="cuda") for _ in self._graphs]
        n = len(self._graphs)
        P = ctypes.c_void_p
        harr = (P * n)(*[g.handle for g in self._graphs])
        carr = (P * n)(*[_ptr(c) for c in self.counts])
        o = _options(**opts)
        self._h = ctypes.c_void_p()
        _check(_lib.gs_plan_3pcf_batch(harr, n, carr, ctypes.byref(o), ctypes.byref(self._h)),
               "gs_plan_3pcf_batch")

    def launch(self, stream=None):
        s = None if stream is None else ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        _check(_lib.gs_plan_launch(self._h, s), "gs_plan_launch")

    def wait(self, stream=None):
        s = None if stream is None else ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        _check(_lib.gs_plan_wait(self._h, s), "gs_plan_wait")
        return self.counts

    def close(self):
        if getattr(self, "_h", None):
            _lib.gs_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
