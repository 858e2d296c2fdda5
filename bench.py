#!/usr/bin/env python
"""Throughput benchmark: binned triangle counts per second on GB300.

Workload (default): 1,000,000 Neyman-Scott points (parents uniform,
Poisson(10) children, Gaussian sigma 2 h^-1Mpc) plus 3,000,000 uniform
randoms in a periodic box L = 1000 h^-1Mpc, FP32 weights U(0.5, 1.5),
rmax = 40 h^-1Mpc in 20 linear bins; DDD and RRR 3pCF, unweighted u64
counts and exact weighted sums. One step = for both catalogues: lattice
quantisation, device graph build, triangle counting (one pass that
produces the counts and the weighted sums). Positions and weights are
resident in HBM when the timed region starts; the graphs (about 5 GB for
the randoms) are larger than L2, so no flush is needed between steps.

Under torchrun every rank processes its own independent realisation
(seeds offset by rank): weak scaling, no collective on the data path.

--impl reference times the CPU oracle (the plain restatement of the
paper's definitions) on a bounded hub sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import catalogs  # noqa: E402

WORKLOAD = "ns1M_L1000_r40_nb20"
METRIC = "binned triplets/s (DDD+RRR 3pCF, counts + exact weighted sums)"
UNIT = "triplets/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle sample")
    ap.add_argument("--no-4pcf", action="store_true",
                    help="skip the secondary 4pCF + parity measurement")
    ap.add_argument("--profile", choices=["count3", "count3w", "count4", "count4w", "pairs",
                                          "equi3w", "mu3", "count4pix"],
                    default=None,
                    help="run one small case of one kernel for an ncu capture (no JSON)")
    ap.add_argument("--variant", type=int, default=0,
                    help="launch variant bits for the --profile case (0 = the library default)")
    ap.add_argument("--no-next", action="store_true",
                    help="skip the connected 4pCF, equilateral and tooling measurements")
    ap.add_argument("--mocks", type=int, default=256,
                    help="lognormal mock catalogues served through the request loop (0 = skip)")
    ap.add_argument("--mock-nmax", type=float, default=4e5)
    ap.add_argument("--mock-grid", type=int, default=256,
                    help="Gaussian-field grid of the lognormal mocks (cells per side)")
    ap.add_argument("--no-ooc", action="store_true",
                    help="skip the out-of-core measurement on the 1e6-point rmax-150 workload")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


KERNEL_VERSION = "k_count3p.v1"  # bump when k_count3 changes; stale captures then report null


KERNEL4_VERSION = "k_count4.v5"  # likewise for k_count4


def _profile_values(name):
    p = os.path.join(ROOT, "profiles", name)
    vals = {}
    if os.path.exists(p):
        for line in open(p):
            if "=" in line and not line.startswith("#"):
                k, v = line.split("=", 1)
                vals[k.strip()] = v.strip()
    return vals


def recorded_traffic():
    """Per-launch DRAM bytes of the counting kernel from the committed ncu
    summary, or None when that capture predates the current kernel."""
    vals = _profile_values("count3_traffic.txt")
    if vals.get("kernel_version") != KERNEL_VERSION:
        return None
    try:
        return float(vals["dram_bytes_per_launch_full_size"])
    except (KeyError, ValueError):
        return None


def recorded_traffic4(edges):
    """Per-launch DRAM bytes of k_count4 scaled from the committed capture by
    the edge count, or None when that capture predates the current kernel."""
    vals = _profile_values("count4_traffic.txt")
    if vals.get("kernel_version") != KERNEL4_VERSION:
        return None
    try:
        return float(vals["dram_bytes_per_launch_profile_case"]) * edges / \
            float(vals["edges_profile_case"])
    except (KeyError, ValueError, ZeroDivisionError):
        return None


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx = float(f[2])
                except ValueError:
                    continue
                for k, nm in enumerate(names):
                    if f[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            os.unlink(self.path)
        except OSError:
            pass
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def load_workload(rank):
    spec = catalogs.WORKLOADS[WORKLOAD]
    off = 1000 * rank
    d = catalogs.draw(WORKLOAD, seed=spec["seed"] + off)
    w_d = catalogs.uniform_weights(spec["n"], seed=spec["weight_seed"] + off)
    pos_r = catalogs.uniform(spec["randoms"], spec["box"], seed=spec["random_seed"] + off)
    w_r = catalogs.uniform_weights(spec["randoms"], seed=spec["weight_seed"] + 7 + off)
    return d, [(d["pos"], w_d), (pos_r, w_r)]


# ----------------------------------------------------------------------------
# CPU oracle arm


# Stand-in for the 3e6 randoms in the oracle's sample: a uniform catalogue
# at the same density (3e-3 per (h^-1 Mpc)^3) in a smaller periodic box,
# whose hubs have the same neighbour statistics (building the oracle's
# graph of all 3e6 randoms takes minutes and about 30 GB of host memory).
RANDOMS_STANDIN_N = 300_000


def randoms_standin():
    spec = catalogs.WORKLOADS[WORKLOAD]
    side = spec["box"] * (RANDOMS_STANDIN_N / spec["randoms"]) ** (1.0 / 3.0)
    box_u = int(round(side * catalogs.LATTICE_PER_MPC))
    side = box_u / catalogs.LATTICE_PER_MPC
    pos = catalogs.uniform(RANDOMS_STANDIN_N, side, seed=spec["random_seed"] + 100)
    w = catalogs.uniform_weights(RANDOMS_STANDIN_N, seed=spec["weight_seed"] + 100)
    return pos, w, box_u, side


class OracleMix:
    """The oracle's 3pCF (counts + exact weighted sums) over the same
    fraction f of the hubs of each catalogue of the step: hubs [0, f N_D) of
    the 1e6-point data catalogue and f N_R hubs at the randoms' density. The
    triangles counted over the time taken is the oracle's rate on the step's
    own mix of clustered and uniform work. Graph builds are not timed."""

    def __init__(self, cats, box_u, edges, nthreads):
        import oracle
        spec = catalogs.WORKLOADS[WORKLOAD]
        self.nd, self.nr = spec["n"], spec["randoms"]
        self.gd = oracle.Graph(oracle.quantize(cats[0][0], box_u, True), box_u, edges,
                               nthreads=nthreads)
        self.wd = cats[0][1]
        pos, self.wr, rbox_u, self.rside = randoms_standin()
        self.gr = oracle.Graph(oracle.quantize(pos, rbox_u, True), rbox_u, edges,
                               nthreads=nthreads)
        self.nthreads = nthreads
        self.f = 1e-3

    def run(self, f):
        kd = max(1, int(f * self.nd))
        kr = min(RANDOMS_STANDIN_N, max(1, int(f * self.nr)))
        t0 = time.perf_counter()
        cd, _ = self.gd.count_3pcf(self.wd, hub_lo=0, hub_hi=kd)
        cr, _ = self.gr.count_3pcf(self.wr, hub_lo=0, hub_hi=kr)
        dt = time.perf_counter() - t0
        return float(cd.sum()) + float(cr.sum()), dt, kd, kr

    def calibrate(self, seconds):
        """Choose f so that one run takes about `seconds`."""
        f = 2e-3
        _, dt, _, _ = self.run(f)
        self.f = min(RANDOMS_STANDIN_N / self.nr, max(1e-4, f * seconds / max(dt, 1e-3)))
        return self.f

    def sample(self, kd, kr):
        return (f"oracle 3pCF (counts + exact weighted sums), same hub fraction of each catalogue: "
                f"hubs [0, {kd}) of the 1e6-point Neyman-Scott data catalogue and [0, {kr}) of "
                f"a {RANDOMS_STANDIN_N}-point uniform catalogue at the randoms' density (periodic "
                f"L = {self.rside:.2f}); query time only")


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    spec, cats = load_workload(0)
    box_u, edges = spec["box_u"], spec["edges_u"]
    nthreads = oracle.default_threads()
    mix = OracleMix(cats, box_u, edges, nthreads)
    # size one step to about budget / (steps + warmup) seconds
    f = mix.calibrate(max(2.0, 150.0 / (args.steps + args.warmup)))
    for _ in range(args.warmup):
        mix.run(f)
    tri, dt = 0.0, 0.0
    for _ in range(args.steps):
        t, d, kd, kr = mix.run(f)
        tri += t
        dt += d
    value = tri / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "hub_fraction": f, "data_hubs_per_step": kd,
                       "random_hubs_per_step": kr},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": mix.sample(kd, kr)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU arm


def run_ours(args):
    import ctypes

    import torch

    import paper_2607_06604_gb300 as gs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    spec, cats = load_workload(rank)
    box_u, edges = spec["box_u"], spec["edges_u"]
    stream = torch.cuda.current_stream()
    dev = [(torch.from_numpy(p).cuda(), torch.from_numpy(w).cuda()) for p, w in cats]
    xyz = [torch.empty((p.shape[0], 3), dtype=torch.int32, device="cuda") for p, _ in dev]
    nconf = gs.gs_num_configs(3, len(edges) - 1)
    counts = [torch.empty(nconf, dtype=torch.uint64, device="cuda") for _ in dev]
    wsums = [torch.empty(nconf, dtype=torch.float64, device="cuda") for _ in dev]
    kms = ctypes.c_double(0.0)
    kernel_ms = []

    def step(record=False):
        for c, (pos, w) in enumerate(dev):
            gs.gs_quantize(pos, box_u, True, out=xyz[c], stream=stream)
            g = gs.gs_build_graph(xyz[c], box_u, edges, stream=stream)
            gs.gs_count_3pcf(g, w, counts=counts[c], wsum=wsums[c], stream=stream, kernel_ms=kms)
            if record and c == 1:
                kernel_ms.append(kms.value)
            g.close()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    tri_step = float(sum(int(c.sum().item()) for c in counts))
    # statistics of the randoms' graph for the roofline (outside the timed region)
    g = gs.gs_build_graph(gs.gs_quantize(dev[1][0], box_u, True), box_u, edges)
    info = gs.gs_graph_info(g)
    g.close()

    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        launches0 = gs.gs_kernel_launches()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            step(record=True)
        t1.record(stream)
        torch.cuda.synchronize()
        launches = gs.gs_kernel_launches() - launches0
    barrier()
    ms = t0.elapsed_time(t1)
    ms_t = torch.tensor([ms], dtype=torch.float64, device="cuda")
    tri_t = torch.tensor([tri_step], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(ms_t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.all_reduce(tri_t, op=torch.distributed.ReduceOp.SUM)
    ms = float(ms_t.item())
    total_tri = float(tri_t.item()) * args.steps
    value = total_tri / (ms / 1e3)

    # End to end through the C ABI with HOST buffers: the pinned host
    # positions go straight to gs_quantize (which copies them in), the
    # pinned host weights to gs_count_3pcf, whose counts and weighted sums
    # come back into pinned host arrays; every step.
    pinned = [(torch.from_numpy(p).pin_memory(), torch.from_numpy(w).pin_memory()) for p, w in cats]
    host_out = [(torch.empty(nconf, dtype=torch.uint64).pin_memory(),
                 torch.empty(nconf, dtype=torch.float64).pin_memory()) for _ in cats]
    h2d = sum(p.numel() * p.element_size() + w.numel() * w.element_size() for p, w in pinned)
    d2h = sum(c.numel() * c.element_size() + s.numel() * s.element_size() for c, s in host_out)

    def step_e2e():
        for c, (pos_h, w_h) in enumerate(pinned):
            gs.gs_quantize(pos_h, box_u, True, out=xyz[c], stream=stream)
            g = gs.gs_build_graph(xyz[c], box_u, edges, stream=stream)
            gs.gs_count_3pcf(g, w_h, counts=host_out[c][0], wsum=host_out[c][1], stream=stream)
            g.close()

    step_e2e()
    e2e_same = all(np.array_equal(host_out[c][0].numpy(), counts[c].cpu().numpy()) and
                   np.array_equal(host_out[c][1].numpy(), wsums[c].cpu().numpy())
                   for c in range(len(cats)))
    barrier()
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    barrier()
    e_s = time.perf_counter() - e0
    e_t = torch.tensor([e_s], dtype=torch.float64, device="cuda")
    if world > 1:
        torch.distributed.all_reduce(e_t, op=torch.distributed.ReduceOp.MAX)
    e2e_value = total_tri / float(e_t.item())

    # Roofline of the dominant kernel (k_count3 on the randoms). Algorithmic
    # bytes per launch, as the scope defines them: 5 bytes (a 4-byte id and a
    # 1-byte bin) per edge for the hub rows once and for every spoke row
    # N+(j) per hub-spoke edge: 5 (E + sum_(i,j) |N+(j)|). A stricter count
    # (4-byte words, spoke rows only up to the merge-walk's exhaustion point)
    # is reported beside it.
    peak, peak_kind = measured_peaks()
    bpe = info["bytes_per_edge"]
    alg_bytes = 5 * (info["edges"] + info["probe_words"])
    strict_bytes = bpe * (info["edges"] + info["walk_words"])
    k_ms = float(np.mean(kernel_ms)) if kernel_ms else float("nan")
    achieved = alg_bytes / (k_ms / 1e3) / 1e9
    traffic = recorded_traffic()
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
            "per_unit": "5 B per edge of the hub row and of every spoke row N+(j)",
            "limiter": "shared-memory pipe (pair tests on staged neighbours, histogram atomics)",
            "kernel": "k_count3p (RRR)", "kernel_ms": k_ms, "alg_bytes_per_launch": alg_bytes,
            "strict_bytes_per_launch": strict_bytes,
            "strict_frac": strict_bytes / (k_ms / 1e3) / 1e9 / peak,
            "triangles_per_launch": float(counts[1].sum().item())}

    if rank != 0:
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        import oracle
        nthreads = oracle.default_threads()
        mix = OracleMix(cats, box_u, edges, nthreads)
        f = mix.calibrate(args.cpu_seconds)
        tri_cpu, dt_cpu, kd, kr = mix.run(f)
        cpu = {"value": tri_cpu / dt_cpu, "unit": UNIT, "cores": nthreads, "kind": "oracle",
               "sample": mix.sample(kd, kr) + f" ({dt_cpu:.1f} s)"}
        del mix
    clocks = clk.summary()
    quad = None
    if not args.no_4pcf:
        quad = measure_4pcf(gs, torch)
    nxt = None if args.no_next else measure_next(gs, torch, dev[1], box_u, edges, k_ms)
    del dev
    torch.cuda.empty_cache()
    ooc = None if args.no_ooc else measure_ooc(gs, torch)
    mocks = measure_mocks(gs, torch, args.mocks, args.mock_nmax, args.mock_grid) \
        if args.mocks else None
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_data": spec["n"], "n_randoms": spec["randoms"],
                       "box": spec["box"], "rmax": spec["rmax"], "nb": spec["nb"],
                       "weights": "fp32 U(0.5,1.5), exact fixed-point sums",
                       "parallelism": f"independent realisation per rank x{world}",
                       "l2": "inputs larger than L2 (randoms' graph "
                             f"{info['edge_slots'] * bpe / 1e9:.1f} GB)"},
            "triangles_per_step": tri_step,
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "results_identical": bool(e2e_same),
                    "path": "pinned host positions, weights and outputs passed to the C ABI"},
            "gpu_launches": int(launches), "clocks": clocks, "quadruplets": quad,
            "mocks": mocks, "out_of_core": ooc, "next_rows": nxt,
            "graph_randoms": {k2: info[k2] for k2 in ("edges", "max_degree", "probe_words",
                                                      "walk_words", "edge_slots")}}
    print(json.dumps(line), flush=True)


def measure_4pcf(gs, torch, runs=2):
    """Quadruplets/s of the parity 4pCF on 2e5 Neyman-Scott points (L=400,
    rmax 30 in 8 bins), plus the pair sweep and disconnected term, with the
    roofline of the counting kernel: algorithmic bytes per launch
    B4 = 5 (E + sum_(i,j) |N+(j)| + sum_(triangles i<j<k) |N+(k)|), the 3pCF
    walk plus the row of every triangle's third vertex that the three-way
    merge of Eq. threeway reads."""
    spec = catalogs.draw("ns200k_L400_r30_nb8")
    box_u, edges = spec["box_u"], spec["edges_u"]
    pos = torch.from_numpy(spec["pos"]).cuda()
    g = gs.gs_build_graph(gs.gs_quantize(pos, box_u, True), box_u, edges)
    like = pos
    gs.gs_count_4pcf_parity(g, like=like)
    import ctypes
    km = ctypes.c_double(0.0)
    ms, kms = [], []
    for _ in range(runs):
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        even, odd = gs.gs_count_4pcf_parity(g, like=like, kernel_ms=km)
        t1.record()
        torch.cuda.synchronize()
        ms.append(t0.elapsed_time(t1))
        kms.append(km.value)
    tet = float(even.sum().item())
    pk = ctypes.c_double(0.0)
    gs.gs_disconnected_4pcf(g, like=like, kernel_ms=pk)
    info = gs.gs_graph_info(g)
    tri, tail = gs.gs_graph_tri_words(g)
    g.close()
    best = min(ms)
    k_ms = min(kms)
    peak, peak_kind = measured_peaks()
    b4 = 5 * (info["edges"] + info["probe_words"] + tail)
    achieved = b4 / (k_ms / 1e3) / 1e9
    return {"workload": "ns200k_L400_r30_nb8", "metric": "binned quadruplets/s (4pCF even+odd)",
            "value": tet / (best / 1e3), "unit": "quadruplets/s", "tetrahedra": tet,
            "triangles": tri, "call_ms": best, "kernel_ms": k_ms, "pair_sweep_ms": pk.value,
            "pair_sweep_gbs": info["edge_slots"] * 4 / (pk.value / 1e3) / 1e9 if pk.value else None,
            "odd_abs_sum": float(odd.abs().sum().item()),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": recorded_traffic4(info["edges"]),
                         "peak_kind": peak_kind,
                         "kernel": "k_count4 (parity)", "alg_bytes_per_launch": b4,
                         "per_unit": "5 B per edge: hub rows, spoke rows, and the row of each "
                                     "triangle's third vertex",
                         "limiter": "instruction issue on shared-memory bit rows (the rows of "
                                    "a hub's neighbourhood are staged once per hub)"}}


def measure_next(gs, torch, randoms, box_u, edges, count3_ms):
    """The rows beyond the core path, each timed with CUDA events after one
    warm-up call: the equilateral and the anisotropic (mu-binned) 3pCF on the
    randoms' graph of the default workload (beside the full 3pCF kernel
    time), the pixelised-direction
    parity 4pCF on the 2e5-point 4pCF workload, the signed-weight connected
    4pCF on 1e5 data + 1e5 randoms, and the configuration tooling."""
    import ctypes

    def timed(fn):
        fn()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        out = fn()
        t1.record()
        torch.cuda.synchronize()
        return out, t0.elapsed_time(t1)

    out = {}
    pos, w = randoms
    g = gs.gs_build_graph(gs.gs_quantize(pos, box_u, True), box_u, edges)
    info = gs.gs_graph_info(g)
    km = ctypes.c_double(0.0)
    (c, _), ms = timed(lambda: gs.gs_count_3pcf_equilateral(g, w, kernel_ms=km))
    words = info["edges"] + info["probe_words"]
    out["equilateral"] = {
        "workload": "3e6 uniform randoms, L=1000, rmax 40, 20 bins, weighted",
        "call_ms": ms, "kernel_ms": km.value, "triangles": float(c.sum().item()),
        "full_3pcf_kernel_ms": count3_ms,
        "alg_bytes_per_launch": 4 * words,
        "achieved_gbs": 4 * words / (km.value / 1e3) / 1e9 if km.value else None}
    # anisotropic 3pCF: 10 mu bins of the triangle normal against the z axis
    kmu = ctypes.c_double(0.0)
    cmu, ms_mu = timed(lambda: gs.gs_count_3pcf_mu(g, 10, like=pos, kernel_ms=kmu))
    tmu = float(cmu.sum().item())
    out["anisotropic_3pcf"] = {
        "workload": "3e6 uniform randoms, L=1000, rmax 40, 20 bins x 10 mu bins, unweighted",
        "call_ms": ms_mu, "kernel_ms": kmu.value, "triangles": tmu,
        "triangles_per_s": tmu / (ms_mu / 1e3), "full_3pcf_kernel_ms": count3_ms}
    g.close()

    # pixelised-direction parity 4pCF on the 2e5-point 4pCF workload
    s4 = catalogs.draw("ns200k_L400_r30_nb8")
    p4 = torch.from_numpy(s4["pos"]).cuda()
    g4 = gs.gs_build_graph(gs.gs_quantize(p4, s4["box_u"], True), s4["box_u"], s4["edges_u"])
    kp = ctypes.c_double(0.0)
    (ev, od), ms = timed(lambda: gs.gs_count_4pcf_parity_pix(g4, like=p4, kernel_ms=kp))
    _, od_exact = gs.gs_count_4pcf_parity(g4, like=p4)
    tet4 = float(ev.sum().item())
    out["parity_pix"] = {
        "workload": "ns200k_L400_r30_nb8", "call_ms": ms, "kernel_ms": kp.value,
        "tetrahedra": tet4, "quadruplets_per_s": tet4 / (ms / 1e3),
        "odd_abs_sum": float(od.abs().sum().item()),
        "odd_abs_sum_exact_channel": float(od_exact.abs().sum().item())}
    g4.close()

    spec = catalogs.draw("ns100k_r100k_L400_r30_nb8")
    bu, e4 = spec["box_u"], spec["edges_u"]
    R = catalogs.uniform(spec["randoms"], spec["box"], spec["random_seed"])
    wd = catalogs.uniform_weights(spec["n"], seed=spec["weight_seed"]).astype(np.float64)
    wr = catalogs.uniform_weights(spec["randoms"], seed=spec["weight_seed"] + 1).astype(np.float64)
    ws = np.concatenate([wd / wd.sum(), -wr / wr.sum()]).astype(np.float32)
    wr1 = (wr / wr.sum()).astype(np.float32)
    U = torch.from_numpy(np.concatenate([spec["pos"], R])).cuda()
    gdr = gs.gs_build_graph(gs.gs_quantize(U, bu, True), bu, e4)
    gr = gs.gs_build_graph(gs.gs_quantize(torch.from_numpy(R).cuda(), bu, True), bu, e4)
    wsd, wrd = torch.from_numpy(ws).cuda(), torch.from_numpy(wr1).cuda()
    kc = ctypes.c_double(0.0)
    res, ms = timed(lambda: gs.gs_connected_4pcf(gdr, wsd, gr, wrd, kernel_ms=kc))
    tet = float(gs.gs_count_4pcf(gdr).sum()) + float(gs.gs_count_4pcf(gr).sum())
    out["connected_4pcf"] = {
        "workload": "ns100k_r100k_L400_r30_nb8", "call_ms": ms, "kernel_ms": kc.value,
        "tetrahedra": tet, "quadruplets_per_s": tet / (ms / 1e3),
        "finite_orbits": int(torch.isfinite(res["zeta_conn"]).sum().item())}
    gdr.close()
    gr.close()

    edges16 = np.array([int(20 * 1024 + b * 2.8125 * 1024) for b in range(17)], dtype=np.int64)
    (mask, kept), ms_cm = timed(lambda: gs.gs_config_mask_cm(16, edges16))
    n16 = gs.gs_num_configs(4, 16)
    rng = np.random.default_rng(0)
    ev = torch.from_numpy(rng.integers(0, 1 << 30, n16).astype(np.uint64)).cuda()
    bmap = torch.from_numpy((np.arange(16) // 2).astype(np.int32)).cuda()
    _, ms_rb = timed(lambda: gs.gs_rebin_4pcf(16, 8, bmap, ev))
    out["tooling"] = {"cm_mask_nb16_ms": ms_cm, "orbits": n16, "realisable": kept,
                      "rebin_4pcf_16_to_8_ms": ms_rb}
    return out


def _one_mock(args):
    n, L, seed, grid = args
    return catalogs.lognormal(int(n), L, seed=seed, grid=grid)


def make_mocks(count, nmax, grid, seed=11):
    """Lognormal mock ensemble: sizes log-uniform in [5e4, nmax], L = 500,
    each catalogue drawn from its own Gaussian field on a grid^3 mesh
    (P(k) ~ k^-1.5, 2 h^-1 Mpc smoothing). Generated on the host in a pool
    of fresh (spawned) worker processes."""
    import multiprocessing as mp
    rng = np.random.Generator(np.random.PCG64(seed))
    sizes = np.exp(rng.uniform(np.log(5e4), np.log(nmax), size=count)).astype(int)
    L = 500.0
    jobs = [(int(n), L, seed * 1000 + k, grid) for k, n in enumerate(sizes)]
    workers = max(1, min(16, (os.cpu_count() or 2) - 1))
    with mp.get_context("spawn").Pool(workers) as pool:
        out = pool.map(_one_mock, jobs, chunksize=1)
    return out, sizes, L


def measure_mocks(gs, torch, count, nmax, grid):
    """The mock-ensemble campaign: 3pCF (rmax 60, 12 bins) of every
    catalogue and, for the first 32, the parity 4pCF (rmax 25, 6 bins).
    (a) one catalogue at a time through the plain API (build, count, free);
    (b) the request loop with every request submitted at once (saturated:
    its throughput is the capacity); (c) the request loop under Poisson
    arrivals at 0.8x that capacity (latency arrival -> result)."""
    L = 500.0
    box_u = int(L * 1024)
    e3 = catalogs.bin_edges_u(0.0, 60.0, 12)
    e4 = catalogs.bin_edges_u(0.0, 25.0, 6)
    t_gen = time.perf_counter()
    mocks, sizes, _ = make_mocks(count, nmax, grid)
    t_gen = time.perf_counter() - t_gen
    xyz = [gs.gs_quantize(p, box_u, True) for p in mocks]
    del mocks
    kinds = [4 if k < 32 else 3 for k in range(count)]
    # a) one catalogue at a time through the plain API; the device time of
    # each call's main kernels is summed to show where the wall time goes
    import ctypes
    km = ctypes.c_double(0.0)
    busy = {"build_ms": 0.0, "count3_ms": 0.0, "count4_ms": 0.0}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain, plain4 = [], {}
    for k, X in enumerate(xyz):
        g = gs.gs_build_graph(X, box_u, e3, kernel_ms=km)
        busy["build_ms"] += km.value
        plain.append(gs.gs_count_3pcf(g, kernel_ms=km))
        busy["count3_ms"] += km.value
        g.close()
        if kinds[k] == 4:
            g4 = gs.gs_build_graph(X, box_u, e4, kernel_ms=km)
            busy["build_ms"] += km.value
            plain4[k] = gs.gs_count_4pcf_parity(g4, kernel_ms=km)
            busy["count4_ms"] += km.value
            g4.close()
    t_plain = time.perf_counter() - t0
    busy_total_s = sum(busy.values()) / 1e3
    tri = float(sum(int(c.sum()) for c in plain))
    tet = float(sum(int(e.sum()) for e, _ in plain4.values()))

    def serve(rate):
        lat, res = [], {}
        rng = np.random.default_rng(5)
        with gs.gs_server() as srv:
            t_start = time.perf_counter()
            tickets = []
            for k, X in enumerate(xyz):
                if rate:
                    time.sleep(rng.exponential(1.0 / rate))
                tickets.append((k, srv.submit(X, box_u, e3, npoint=3)))
                if kinds[k] == 4:
                    tickets.append((-1 - k, srv.submit(X, box_u, e4, npoint=4)))
            for k, t in tickets:
                c, o, ws, info = srv.wait(t)
                lat.append(info["t_done"] - info["t_submit"])
                res[k] = (c, o)
            span = time.perf_counter() - t_start
        return span, np.array(lat), res

    def identical(res):
        ok = all(np.array_equal(res[k][0], plain[k]) for k in range(count))
        return ok and all(np.array_equal(res[-1 - k][0], e) and np.array_equal(res[-1 - k][1], o)
                          for k, (e, o) in plain4.items())

    t_sat, lat_sat, res = serve(0.0)
    same = identical(res)
    capacity = count / t_sat
    t_poi, lat_poi, res2 = serve(0.8 * capacity)
    same = same and identical(res2)
    return {"catalogues": count, "n_range": [int(sizes.min()), int(sizes.max())],
            "points": int(sizes.sum()), "grid": grid,
            "box": L, "rmax3": 60.0, "nb3": 12, "rmax4": 25.0, "nb4": 6, "also_4pcf": min(32, count),
            "triangles": tri, "tetrahedra": tet, "host_generation_s": t_gen,
            "one_at_a_time_s": t_plain, "one_at_a_time_catalogues_per_s": count / t_plain,
            "one_at_a_time_kernel_ms": busy,
            "one_at_a_time_kernel_busy_fraction": busy_total_s / t_plain,
            "served_saturated_s": t_sat, "served_catalogues_per_s": capacity,
            "speedup_vs_one_at_a_time": t_plain / t_sat,
            "poisson_rate_per_s": 0.8 * capacity, "poisson_span_s": t_poi,
            "latency_p50_s": float(np.percentile(lat_poi, 50)),
            "latency_p99_s": float(np.percentile(lat_poi, 99)),
            "saturated_latency_p50_s": float(np.percentile(lat_sat, 50)),
            "saturated_latency_p99_s": float(np.percentile(lat_sat, 99)),
            "results_identical_to_single_calls": bool(same)}


def measure_ooc(gs, torch):
    """Out-of-core overhead on 1e6 Neyman-Scott points (sigma 5) in an open
    box L = 1494, rmax 150 in 15 bins, under a 16 GB device graph budget and
    with forced window counts: t(windows) / t(resident) - 1."""
    import ctypes
    spec = catalogs.draw("ns1M_open_L1494_r150_nb15")
    box_u, edges = spec["box_u"], spec["edges_u"]
    X = gs.gs_quantize(torch.from_numpy(spec["pos"]).cuda(), box_u, False)
    out = {"workload": "ns1M_open_L1494_r150_nb15", "budget_bytes": 16 << 30}
    base = None
    for label, kw in (("resident", {}), ("budget_16GB", {"budget": 16 << 30}),
                      ("W2", {"force_windows": 2}), ("W4", {"force_windows": 4}),
                      ("W8", {"force_windows": 8})):
        g = gs.gs_build_graph(X, 0, edges, **kw)
        info = gs.gs_graph_info(g)
        km = ctypes.c_double(0.0)
        t0 = time.perf_counter()
        c = gs.gs_count_3pcf(g, like=X, kernel_ms=km)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if base is None:
            base = c.cpu().numpy()
            out["edges"] = info["edges"]
            out["graph_bytes"] = info["edge_slots"] * 4
            out["triangles"] = float(base.sum())
        same = bool(np.array_equal(c.cpu().numpy(), base))
        out[label] = {"windows": info["windows"], "query_s": dt, "kernel_ms": km.value,
                      "identical": same}
        g.close()
    for label in ("budget_16GB", "W2", "W4", "W8"):
        out[label]["overhead"] = out[label]["query_s"] / out["resident"]["query_s"] - 1.0
    return out


def run_profile(args):
    """One small case per kernel, sized above L2 but a few GB at most."""
    import torch

    import paper_2607_06604_gb300 as gs
    torch.cuda.set_device(0)
    if args.profile in ("count3", "count3w", "pairs", "equi3w", "mu3"):
        # 1e6 uniform points at the randoms' density (3e-3 per (h^-1 Mpc)^3),
        # rmax 40 in 20 bins: a 1.6 GB graph
        L = 693.0
        box_u = int(L * 1024)
        pos = torch.from_numpy(catalogs.uniform(1_000_000, L, seed=5)).cuda()
        edges = catalogs.bin_edges_u(0.0, 40.0, 20)
        g = gs.gs_build_graph(gs.gs_quantize(pos, box_u, True), box_u, edges)
        w = torch.from_numpy(catalogs.uniform_weights(1_000_000, seed=6)).cuda()
        for _ in range(2):
            if args.profile == "count3":
                gs.gs_count_3pcf(g, like=pos, variant=args.variant)
            elif args.profile == "count3w":
                gs.gs_count_3pcf(g, w, variant=args.variant)
            elif args.profile == "equi3w":
                gs.gs_count_3pcf_equilateral(g, w)
            elif args.profile == "mu3":
                gs.gs_count_3pcf_mu(g, 10, like=pos)
            else:
                gs.gs_disconnected_4pcf(g, like=pos, zeta=False)
    else:
        # 1e5 Neyman-Scott points at the 4pCF workload's density (L=317)
        L = 317.0
        box_u = int(L * 1024)
        pos = torch.from_numpy(catalogs.neyman_scott(100_000, L, seed=6, sigma=2.0)).cuda()
        edges = catalogs.bin_edges_u(0.0, 30.0, 8)
        g = gs.gs_build_graph(gs.gs_quantize(pos, box_u, True), box_u, edges)
        # count4w: signed weights (40% negative), as in the connected estimator
        rng = np.random.default_rng(7)
        w = torch.from_numpy((catalogs.uniform_weights(100_000, seed=8) *
                              np.where(rng.random(100_000) < 0.4, -1.0, 1.0))
                             .astype(np.float32)).cuda()
        for _ in range(2):
            if args.profile == "count4w":
                gs.gs_count_4pcf_parity(g, w)
            elif args.profile == "count4pix":
                gs.gs_count_4pcf_parity_pix(g, like=pos)
            else:
                gs.gs_count_4pcf_parity(g, like=pos)
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "info": gs.gs_graph_info(g)}))


def main():
    args = parse()
    if args.profile:
        run_profile(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
    if int(os.environ.get("WORLD_SIZE", 1)) > 1:
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
