#!/usr/bin/env python
"""Benchmark of the anisotropic-3PCF hot path on GB300 (one JSON line on rank 0).

Workload (default): the clustered catalog -- N = 2,000,000 points in a
periodic cube of side 1500 Mpc/h, 60% uniform and 40% in sigma = 5 Mpc/h
Gaussian blobs about 10,000 uniform centres, FP32 positions, weights
U(0.5, 1.5), Rmax = 200, 10 linear bins on [0, 200], lmax = 10, LOS = z.
A step is one full forward: index build, pair stage (all pairs within Rmax
binned, Y_lm, a_lm), the zeta contraction and the FP64 reduction.

Reported: ``value`` = accepted pairs per second (whole job), ``zeta_tflops`` =
algorithmic contraction rate, both for the split-BF16 tensor-core form (the
default) with the plain-FP32 form beside it; ``roofline`` for the dominant
kernel (the pair stage, bound by the FP32 FMA pipe); ``e2e`` through the C ABI
from pinned host buffers; ``cpu_baseline`` = the FP64 oracle on a bounded sample.

``--impl reference`` times the FP64 oracle itself on the host cores (bounded
sample of the same workload per step).  N > 1 GPUs run independent replicas
(the path is one GPU by design); value = pairs of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pairs/s through a_lm + zeta TFLOP/s, FP32 vs split-TC form at 1e-4 rel err"
WORKLOAD = ("clustered N=2,000,000, periodic cube L=1500 Mpc/h, 60% uniform + 40% sigma=5 blobs "
            "about 10,000 centres, FP32 pos, w~U(0.5,1.5), Rmax=200, 10 bins, lmax=10, LOS=z")
# Algorithmic FP32 flops per accepted pair of the pair stage at lmax = L:
# r^2 and rhat (8), w (x+iy)^m (2 + 6(L-1)), the Legendre-type recurrence
# (3 L(L-1)/2), the m = 0 accumulation (L + 2(L+1) with the leading terms)
# and the m > 0 complex accumulation (4 L(L+1)/2): 451 at L = 10.
def pair_flops(L: int) -> int:
    return 8 + (2 + 6 * (L - 1)) + 3 * L * (L - 1) // 2 + L + 2 * (L + 1) + 4 * L * (L + 1) // 2


def zeta_flops_per_primary(nbins: int, L: int) -> int:
    # Hermitian upper triangle, complex MAC = 8 flop: 4 sum_m K_m (K_m + 1)
    return sum(4 * (nbins * (L + 1 - m)) * (nbins * (L + 1 - m) + 1) for m in range(L + 1))


# Executed FP32 flops per pair of the accumulate kernel (Chebyshev form, FMA = 2):
# T_k recurrence 2(L-1), m = 0 sums 2L + 1, m >= 1 terms 2 L + 4 L (L - 1) / 2 x 2,
# (x + iy)^m 6 (L - 1) + 2, separation and unit vector 12.
def accum_exec_flops(L: int) -> int:
    if L == 0:
        return 13
    return 2 * (L - 1) + (2 * L + 1) + 2 * L + 4 * (L * (L + 1) // 2 - L) + 6 * (L - 1) + 2 + 12


# DRAM bytes of one k_accum launch per primary, from the ncu capture summarised
# in profiles/k_accum_clustered_200k_L696.md (17.60 GB for 200,000 primaries,
# Lambda = 10); a full-size launch is scaled by its primaries.
ACCUM_DRAM_BYTES_PER_PRIMARY = 17.60e9 / 200000


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if "Active" in r[5 + k]
                          and not r[5 + k].startswith("Not")})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(t: float, device, ws: int) -> float:
    """The slowest rank's step time (all ranks take part; one rank: t)."""
    if ws <= 1:
        return t
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t], device=device, dtype=torch.float64)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(pairs_per_rank: float, ws: int, t_max: float) -> float:
    """Whole-job pairs/s of ws replicas that each processed pairs_per_rank."""
    return ws * pairs_per_rank / t_max


def make_catalog(args):
    from paper_1709_00086_gb300 import catalogs
    if args.workload == "clustered2m":
        return catalogs.clustered_2m(n=args.n or 2_000_000, box=args.box or 1500.0)
    if args.workload == "uniform20k":
        return catalogs.plain_uniform(n=args.n or 20000)
    raise SystemExit("unknown workload")


def oracle_sample(cat, nprim: int):
    """Time the FP64 oracle on nprim primaries (all points secondaries)."""
    import oracle
    pos = cat.pos.astype(np.float64)
    w = cat.w.astype(np.float64)
    rng = np.random.default_rng(123)
    prim = rng.choice(cat.n, size=nprim, replace=False)
    order = np.concatenate([prim, np.setdiff1d(np.arange(cat.n), prim)])
    t0 = time.perf_counter()
    z, c = oracle.zeta(pos[order], w[order], cat.box, cat.nbins, cat.rmin, cat.rmax, cat.lmax,
                       los_mode=cat.los_mode, n_primary=nprim)
    dt = time.perf_counter() - t0
    return int(c.sum()), dt


def run_reference(args):
    ws, rank, _ = dist_info()
    if rank != 0:
        return
    cat = make_catalog(args)
    cores = os.cpu_count()
    per = []
    pairs_tot = 0
    for s in range(args.warmup + args.steps):
        pairs, dt = oracle_sample(cat, args.ref_primaries)
        if s >= args.warmup:
            per.append(dt)
            pairs_tot += pairs
    t = sum(per)
    val = pairs_tot / t
    sample = "%d random primaries of the workload per step (all %d points secondaries)" % (
        args.ref_primaries, cat.n)
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": "pairs/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / len(per),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": WORKLOAD, "form": "FP64 CPU oracle"},
           "cpu_baseline": {"value": val, "unit": "pairs/s", "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def measure_batch(steps: int, warmup: int) -> dict:
    """The batched workload (64 catalogs, sizes log-uniform in [1e3, 1e6], periodic L = 600,
    Rmax = 150, 12 bins, lmax = 8): one compute_batch per step, replayed from a captured CUDA
    graph, against the same call uncaptured."""
    import torch
    import paper_1709_00086_gb300 as g3
    from paper_1709_00086_gb300 import catalogs
    dev = torch.device("cuda", torch.cuda.current_device())
    cats = catalogs.batched(64, seed=3)
    plan = g3.Plan(**cats[0].params())
    pos = torch.from_numpy(np.concatenate([c.pos for c in cats])).to(dev)
    w = torch.from_numpy(np.concatenate([c.w for c in cats])).to(dev)
    offs = np.cumsum([0] + [c.n for c in cats])
    zb = torch.empty((len(cats), plan.zsize, 2), dtype=torch.float64, device=dev)
    cb = torch.empty((len(cats), plan.nbins), dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream()
    res = {}
    for graph in (True, False):
        for _ in range(warmup):
            plan.compute_batch(pos, w, offs, graph=graph, out=zb, counts_out=cb)
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.compute_batch(pos, w, offs, graph=graph, out=zb, counts_out=cb, sync=False)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        plan.status()
        res[graph] = float(np.mean(ms))
    st = plan.stats()
    pairs = float(cb.sum().item())
    # the project autotuner on the largest catalog (whose pairs dominate), through its
    # on-disk cache, then the graph replay again with the tuned grid
    import tempfile
    big = max(range(len(cats)), key=lambda k: cats[k].n)
    sl = slice(int(offs[big]), int(offs[big + 1]))
    t0 = time.perf_counter()
    tune = plan.autotune_cached(pos[sl], w[sl], os.path.join(tempfile.gettempdir(), "g3pcf_tune.txt"))
    tune["seconds"] = time.perf_counter() - t0
    for _ in range(warmup):
        plan.compute_batch(pos, w, offs, graph=True, out=zb, counts_out=cb)
    torch.cuda.synchronize()
    ms = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.compute_batch(pos, w, offs, graph=True, out=zb, counts_out=cb, sync=False)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    plan.status()
    tuned_ms = float(np.mean(ms))
    out = {"workload": "batched: 64 uniform catalogs, sizes log-uniform in [1e3, 1e6] (%d points), "
                       "periodic L=600, Rmax=150, 12 bins, lmax=8, LOS=z" % int(offs[-1]),
           "pairs_per_step": pairs, "graph_ms_per_step": res[True], "graph_pairs_per_s": pairs / (res[True] / 1e3),
           "uncaptured_ms_per_step": res[False], "uncaptured_pairs_per_s": pairs / (res[False] / 1e3),
           "contract_ms": st["contract_ms"], "pair_ms": st["pair_ms"],
           "zeta_tflops": zeta_flops_per_primary(12, 8) * int(offs[-1]) / (st["contract_ms"] / 1e3) / 1e12,
           "tuned": {"settings": tune, "graph_ms_per_step": tuned_ms,
                     "graph_pairs_per_s": pairs / (tuned_ms / 1e3),
                     "vs_default": res[True] / tuned_ms}}
    del plan, pos, w, zb, cb
    torch.cuda.empty_cache()
    return out


def run_batch(args):
    """--workload batch64: the batched workload as the JSON line's own value."""
    b = measure_batch(args.steps, args.warmup)
    out = {"metric": METRIC, "value": b["graph_pairs_per_s"], "unit": "pairs/s", "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": b["graph_ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": b["workload"], "form": "split-BF16 tensor-core contraction, CUDA-graph replay",
                      "pairs_per_step": b["pairs_per_step"], "parallelism": "single GPU"},
           "uncaptured": {"ms_per_step": b["uncaptured_ms_per_step"], "value": b["uncaptured_pairs_per_s"]},
           "tuned": b["tuned"]}
    print(json.dumps(out), flush=True)


def measure_forward(cat, steps: int, warmup: int) -> dict:
    """Plain forwards of one catalog, split-BF16 tensor-core and plain-FP32 contraction."""
    import torch
    import paper_1709_00086_gb300 as g3
    dev = torch.device("cuda", torch.cuda.current_device())
    plan = g3.Plan(**cat.params())
    pos = torch.from_numpy(cat.pos).to(dev)
    w = torch.from_numpy(cat.w).to(dev)
    stream = torch.cuda.current_stream()
    res = {}
    for fp32 in (False, True):
        for _ in range(warmup):
            plan.compute(pos, w, fp32_contraction=fp32, with_counts=False)
        ms, st = [], []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.compute(pos, w, fp32_contraction=fp32, with_counts=False, sync=False)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            st.append(plan.stats())
        plan.status()
        t = float(np.mean(ms))
        con = float(np.mean([x["contract_ms"] for x in st]))
        pairs = st[-1]["pairs"]
        res["fp32" if fp32 else "tc"] = {
            "ms_per_step": t, "pairs_per_s": pairs / (t / 1e3), "contract_ms": con,
            "contract_share": con / t, "pair_ms": float(np.mean([x["pair_ms"] for x in st])),
            "zeta_tflops": zeta_flops_per_primary(cat.nbins, cat.lmax) * st[-1]["primaries"] / (con / 1e3) / 1e12}
    res["pairs_per_step"] = pairs
    # the tensor-core form replayed from a CUDA graph (passes planned on the device:
    # no host round trip and no per-kernel launch cost inside the step); the same
    # output buffer every call, so that every call after the first replays
    zb = torch.empty((plan.zsize, 2), dtype=torch.float64, device=dev)
    for _ in range(max(warmup, 2)):
        plan.compute(pos, w, with_counts=False, graph=True, out=zb)
    ms = []
    for _ in range(steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        plan.compute(pos, w, with_counts=False, sync=False, graph=True, out=zb)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    plan.status()
    tg = float(np.mean(ms))
    res["tc"]["graph_ms_per_step"] = tg
    res["tc"]["graph_pairs_per_s"] = pairs / (tg / 1e3)
    del plan, pos, w
    torch.cuda.empty_cache()
    return res


def measure_adjoint(dev, stream, n: int = 0, list_bytes: int = 0) -> dict:
    """The differentiation workload (clustered N = 500,000, L = 800, Rmax = 120, 8 bins,
    lmax = 6): forward with multipoles kept, then g3pcf_backward, in the default
    double-float gradient arithmetic and in the FP32 form."""
    import torch
    import paper_1709_00086_gb300 as g3
    from paper_1709_00086_gb300 import catalogs as cats
    dcat = cats.differentiation(n=n) if n > 0 else cats.differentiation()
    dpos = torch.from_numpy(dcat.pos).to(dev)
    dwt = torch.from_numpy(dcat.w).to(dev)
    out = {"workload": "clustered N=%d, periodic L=800, Rmax=120, 8 bins, lmax=6" % dcat.n}
    for prec, key in ((0, "double_float"), (1, "fp32")):
        dplan = g3.Plan(**dcat.params())
        dplan.set_option(g3.OPT_GRAD_PRECISION, prec)
        if list_bytes > 0:
            dplan.set_option(g3.OPT_LIST_BYTES, list_bytes)
        rng = np.random.default_rng(5)
        dz = torch.from_numpy(rng.normal(size=(dplan.zsize, 2))).to(dev)
        fwd_ms, bwd_ms = [], []
        for k in range(3):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            dplan.compute(dpos, dwt, keep_alm=True, with_counts=False, fp32_contraction=True)
            e1.record(stream)
            dplan.backward(dz)
            e2.record(stream)
            e2.synchronize()
            if k > 0:
                fwd_ms.append(e0.elapsed_time(e1))
                bwd_ms.append(e1.elapsed_time(e2))
        dpairs = dplan.stats()["pairs"]
        out["pairs"] = dpairs
        out[key] = {"forward_ms": float(np.mean(fwd_ms)), "backward_ms": float(np.mean(bwd_ms)),
                    "backward_pairs_per_s": dpairs / (float(np.mean(bwd_ms)) / 1e3)}
        del dplan
    out["forward_ms"] = out["double_float"]["forward_ms"]
    out["backward_ms"] = out["double_float"]["backward_ms"]
    del dpos, dwt
    torch.cuda.empty_cache()
    return out


def measure_large(dev) -> dict:
    """One forward of the large radial workload (N = 5e7 clustered, open L = 3000, radial LOS,
    Rmax = 200, 10 bins, lmax = 10), after one untimed forward."""
    import torch
    import paper_1709_00086_gb300 as g3
    from paper_1709_00086_gb300 import catalogs as cats
    cat = cats.large_radial()
    plan = g3.Plan(**cat.params())
    pos = torch.from_numpy(cat.pos).to(dev)
    w = torch.from_numpy(cat.w).to(dev)
    stream = torch.cuda.current_stream()
    plan.compute(pos, w, with_counts=False)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.compute(pos, w, with_counts=False, sync=False)
    e1.record(stream)
    e1.synchronize()
    plan.status()
    st = plan.stats()
    ms = e0.elapsed_time(e1)
    out = {"workload": "clustered N=5e7, open cube L=3000, radial LOS from the centre, Rmax=200, 10 bins, lmax=10",
           "forward_ms": ms, "pairs": st["pairs"], "pairs_per_s": st["pairs"] / (ms / 1e3),
           "pair_ms": st["pair_ms"], "contract_ms": st["contract_ms"], "list_passes": st["list_passes"]}
    del plan, pos, w
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    import paper_1709_00086_gb300 as g3
    ws, rank, local = dist_info()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cat = make_catalog(args)
    plan = g3.Plan(**cat.params())
    if args.list_bytes > 0:  # cap the pair-list pool (small-footprint profiling runs)
        plan.set_option(g3.OPT_LIST_BYTES, args.list_bytes)
    pos = torch.from_numpy(cat.pos).to(dev)
    w = torch.from_numpy(cat.w).to(dev)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    L, B = cat.lmax, cat.nbins

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(fp32: bool, steps: int, warmup: int, sampler=None):
        z = None
        for _ in range(warmup):
            z, _ = plan.compute(pos, w, fp32_contraction=fp32, with_counts=False, sync=False)
        plan.status()
        torch.cuda.synchronize()
        barrier()
        if sampler:
            sampler.start()
        ms, st = [], []
        for _ in range(steps):
            flush.fill_(1.0)  # evict L2 between steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            z, _ = plan.compute(pos, w, fp32_contraction=fp32, with_counts=False, sync=False)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            st.append(plan.stats())
        plan.status()
        torch.cuda.synchronize()
        barrier()
        clocks = sampler.stop() if sampler else None
        return z, ms, st, clocks

    sampler = ClockSampler(local) if rank == 0 else None
    z_tc, ms_tc, st_tc, clocks = timed(False, args.steps, args.warmup, sampler)
    z_32, ms_32, st_32, _ = timed(True, max(2, args.steps // 2), 1)
    # isotropic Legendre 3PCF epilogue (g3pcf_isotropic) on the step's zeta
    iso_ms = []
    for k in range(4):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g3.isotropic(z_tc, B, L)
        e1.record(stream)
        e1.synchronize()
        if k > 0:
            iso_ms.append(e0.elapsed_time(e1))
    pairs = st_tc[-1]["pairs"]
    nprim = st_tc[-1]["primaries"]
    t_step = float(np.mean(ms_tc)) / 1e3
    t_max = max_over_ranks(t_step, dev, ws)
    value = job_value(pairs, ws, t_max)
    pair_ms = float(np.mean([s["pair_ms"] for s in st_tc]))
    con_tc = float(np.mean([s["contract_ms"] for s in st_tc]))
    con_32 = float(np.mean([s["contract_ms"] for s in st_32]))
    zf = zeta_flops_per_primary(B, L) * nprim
    diff = (z_tc - z_32).abs().max().item() / max(z_32.abs().max().item(), 1e-300)

    # end to end through the C ABI from pinned host buffers
    hpos = torch.from_numpy(cat.pos).pin_memory()
    hw = torch.from_numpy(cat.w).pin_memory()
    hz = torch.empty((plan.zsize, 2), dtype=torch.float64).pin_memory()
    dpos = torch.empty_like(pos)
    dw = torch.empty_like(w)
    zbuf = torch.empty((plan.zsize, 2), dtype=torch.float64, device=dev)
    e2e_ms = []
    for k in range(args.warmup + max(2, args.steps // 2)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dpos.copy_(hpos, non_blocking=True)
        dw.copy_(hw, non_blocking=True)
        plan.compute(dpos, dw, with_counts=False, out=zbuf)
        hz.copy_(zbuf, non_blocking=True)
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_val = ws * pairs / (float(np.mean(e2e_ms)) / 1e3)

    # the other measured workloads (one GPU only): the plain 20,000-point catalog, the
    # batched 64 catalogs, the differentiation workload's adjoint and, on request, the
    # 50-million-point radial catalog
    adj = None
    other = {}
    if ws == 1:
        if not args.no_adjoint:
            adj = measure_adjoint(dev, stream, args.adjoint_n, args.list_bytes)
        if not args.no_other:
            from paper_1709_00086_gb300 import catalogs as cats
            other["plain_uniform_20k"] = measure_forward(cats.plain_uniform(), max(3, args.steps), args.warmup)
            other["batched_64"] = measure_batch(2, 1)
        if args.large:
            other["large_radial_50m"] = measure_large(dev)

    if rank != 0:
        return
    pk = peaks()
    clk_max = float(pk.get("sm_max_mhz", 2070.0))
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    nominal = 2.0 * 128 * n_sm * clk_max * 1e6 / 1e12  # TFLOP/s, FMA = 2 flop
    fp32_peak = g3.fp32_peak_tflops()
    accum_ms = float(np.mean([s["accum_ms"] for s in st_tc]))
    scan_ms = float(np.mean([s["scan_ms"] for s in st_tc]))
    n_acc = int(st_tc[-1]["accum_launches"]) or 1
    achieved = pairs * pair_flops(L) / (accum_ms / 1e3) / 1e12
    executed = pairs * accum_exec_flops(L) / (accum_ms / 1e3) / 1e12
    out = {
        "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "form": "split-BF16 tensor-core contraction",
                   "pairs_per_step": pairs, "primaries": nprim,
                   "candidates_per_step": st_tc[-1]["candidates"],
                   "l2": "256 MB buffer written between timed steps; per-step working set > L2",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "zeta_tflops": zf / (con_tc / 1e3) / 1e12,
        "stage_ms": {"index": float(np.mean([s["index_ms"] for s in st_tc])), "pair": pair_ms,
                     "pair_scan": scan_ms, "pair_accum": accum_ms,
                     "contract": con_tc, "reduce": float(np.mean([s["reduce_ms"] for s in st_tc])),
                     "isotropic_epilogue": float(np.mean(iso_ms))},
        "fp32_form": {"ms_per_step": float(np.mean(ms_32)), "value": pairs / (np.mean(ms_32) / 1e3),
                      "contract_ms": con_32, "zeta_tflops": zf / (con_32 / 1e3) / 1e12,
                      "max_rel_diff_vs_tc": diff},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak,
                     "traffic": ACCUM_DRAM_BYTES_PER_PRIMARY * nprim / n_acc if L == 10 else None,
                     "kernel": "k_accum<%d> (FP32 FMA pipe), %d launches per step, %.2f ms per launch"
                               % (L, n_acc, accum_ms / n_acc),
                     "peak_source": "measured: g3pcf_fp32_peak FMA-chain probe on this GPU "
                                    "(nominal 2 x 128 lanes x %d SMs x %.0f MHz = %.1f)" % (n_sm, clk_max, nominal),
                     "flops_per_pair": pair_flops(L),
                     "executed_flops_per_pair": accum_exec_flops(L),
                     "executed_tflops": executed,
                     "frac_executed": executed / fp32_peak,
                     # the whole pair stage (candidate scan + accumulate), algorithmic and executed
                     "pair_stage": {"ms": pair_ms,
                                    "achieved": pairs * pair_flops(L) / (pair_ms / 1e3) / 1e12,
                                    "frac": pairs * pair_flops(L) / (pair_ms / 1e3) / 1e12 / fp32_peak,
                                    "frac_executed": pairs * accum_exec_flops(L) / (pair_ms / 1e3) / 1e12
                                                     / fp32_peak}},
        "e2e": {"value": e2e_val, "unit": "pairs/s",
                "h2d_bytes_per_step": int(hpos.numel() * 4 + hw.numel() * 4),
                "d2h_bytes_per_step": int(hz.numel() * 8)},
        "adjoint": adj,
        "other_workloads": other,
        "clocks": clocks,
        "gpu_launches": int(st_tc[-1]["launches"]) * args.steps,
    }
    if not args.no_cpu_baseline:
        pr, dt = oracle_sample(cat, args.cpu_primaries)
        out["cpu_baseline"] = {"value": pr / dt, "unit": "pairs/s", "cores": os.cpu_count(),
                               "kind": "oracle",
                               "sample": "%d random primaries of the workload, all %d points as "
                                         "secondaries, %.1f s" % (args.cpu_primaries, cat.n, dt)}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="clustered2m",
                    help="clustered2m (the benchmark), uniform20k, or batch64 (graph-replayed batch)")
    ap.add_argument("--n", type=int, default=0, help="override N (profiling cases)")
    ap.add_argument("--box", type=float, default=0.0, help="override the box side (profiling cases)")
    ap.add_argument("--cpu-primaries", type=int, default=300)
    ap.add_argument("--ref-primaries", type=int, default=60)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint timing")
    ap.add_argument("--no-other", action="store_true", help="skip the 20k and batched workloads")
    ap.add_argument("--list-bytes", type=int, default=0, help="pair-list pool of the main plan in bytes (0: automatic)")
    ap.add_argument("--adjoint-n", type=int, default=0, help="override N of the differentiation workload (profiling cases)")
    ap.add_argument("--large", action="store_true", help="also time one forward of the 50M radial workload")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch64":
        run_batch(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
