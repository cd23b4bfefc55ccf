#!/usr/bin/env python
"""Benchmark of the b-tree neighbour search (arXiv:1910.02639) on GB300.

One step = the whole hot path over one particle set: BuildTree (bounding box,
per-level sub-cell histograms / ratio test / scan / scatter, warp-level
sub-trees) + FindNeighbors fused with the M4 density (walk, gather, sort,
test, ordered capped rows).  Default workload: the jittered lattice slab of
1e7 particles (400 x 250 x 100, spacing 1, jitter +-0.1, h = 1.5, masses 1/N),
ngmax 256.  Before timing, the autotuner picks this set's bucket size, beta,
work-unit size and find block shape (none changes a result; `config` names
the choice, `default_params` times the untuned s = 16 default beside it).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  `value` = neighbour pairs (sum of uncapped
counts) per second over all ranks, inputs resident in HBM; `e2e` = the same
metric with the inputs copied from pinned host memory and the lists, counts
and densities copied back inside the timed region.  With --impl reference the
CPU oracle is timed instead (a bounded sample, on the host cores).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "neighbor pairs/s (build+find) at 1e7 particles; batched vs plain; p99 latency ms"
UNIT = "pairs/s"
FALLBACK_HBM_GBS = 6800.0


# ---------------------------------------------------------------- workload
def make_workload(name: str):
    from paper_1910_02639_gb300 import workloads as wl
    if name == "slab1e7":
        s = wl.jittered_slab(400, 250, 100, jitter=0.1, h=1.5, seed=1913)
        cfg = dict(workload="jittered_slab_1e7", n=s.n, lattice=[400, 250, 100], jitter=0.1,
                   h=1.5, masses="1/N", bucket_size=16, alpha=0.5, beta=0.5, ngmax=256)
    elif name == "slab2e6":
        s = wl.jittered_slab(200, 100, 100, jitter=0.1, h=1.5, seed=1916)
        cfg = dict(workload="jittered_slab_2e6", n=s.n, lattice=[200, 100, 100], jitter=0.1,
                   h=1.5, masses="1/N", bucket_size=16, alpha=0.5, beta=0.5, ngmax=256)
    elif name == "uniform32k":
        s = wl.uniform_cube(32768, seed=1911)
        cfg = dict(workload="uniform_cube_32768", n=s.n, target_neighbours=100,
                   bucket_size=16, alpha=0.5, beta=0.5, ngmax=256)
    elif name == "evrard1e6":
        s = wl.evrard(1_000_000, seed=1912)
        cfg = dict(workload="evrard_1e6", n=s.n, target_neighbours=100, bucket_size=16,
                   alpha=0.5, beta=0.5, ngmax=512)
    else:
        raise SystemExit(f"unknown workload {name}")
    return s, cfg


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def find_kernel_sha() -> str:
    h = hashlib.sha256()
    for f in ("bt_find.cu", "bt_sort.cuh", "bt_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1910_02639_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _profile_kv(workload: str):
    """Machine-readable lines of the committed ncu summary of the find
    kernel, if it was taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", f"k_find_{workload}.md")
    if not os.path.exists(p):
        return None
    kv = {}
    for line in open(p):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            kv[k.strip()] = v.strip()
    return kv if kv.get("source_sha") == find_kernel_sha() else None


def profiled_traffic(workload: str):
    """DRAM bytes per launch of the find kernel (ncu, scaled to the workload)."""
    kv = _profile_kv(workload)
    try:
        return float(kv["dram_bytes_per_launch_scaled"]) if kv else None
    except (KeyError, ValueError):
        return None


def profiled_warp_insts(workload: str):
    """Warp instructions per launch of the find kernel (ncu, scaled)."""
    kv = _profile_kv(workload)
    try:
        return float(kv["warp_insts_per_launch_scaled"]) if kv else None
    except (KeyError, ValueError):
        return None


def issue_peak(sm_mhz):
    """Peak warp-instruction issue rate: 152 SMs x 4 schedulers x 1 per clock."""
    return 152 * 4 * (sm_mhz or 2070.0) * 1e6


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = [l for (t, l) in self.lines if t0 <= t <= t1] or [l for (_, l) in self.lines]
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            f = [x.strip() for x in r.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- dist
def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        return dist, dist.get_rank(), ws
    return None, 0, 1


def barrier(dist, dev):
    import torch
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier(device_ids=[dev.index])


def reduce_max(dist, v, dev):
    if not dist:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- GPU arm
def run_gpu(args):
    import numpy as np
    import torch

    import paper_1910_02639_gb300 as bt

    dist, rank, ws = dist_init()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    s, cfg = make_workload(args.workload)
    n, ngmax, sb = s.n, cfg["ngmax"], cfg["bucket_size"]
    cfg.update(parallelism="replicas" if ws > 1 else "single",
               l2="no flush: positions (16 B x n) and lists (4 B x ngmax x n) exceed the 129 MB L2",
               density="M4 cubic spline fused into the find pass")
    stream = torch.cuda.current_stream(dev)
    x, y, z, h, m = (torch.from_numpy(a).to(dev) for a in (s.x, s.y, s.z, s.h, s.m))
    nb = torch.empty(n * ngmax, dtype=torch.int32, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev)
    rho = torch.empty(n, dtype=torch.float32, device=dev)
    tree = None

    # ---- parameters: the autotuner's choice for this set (bucket size, beta,
    # work-unit size, find block shape); none of them changes a result
    params = dict(bucket_size=sb, alpha=cfg["alpha"], beta=cfg["beta"])
    tune_s = 0.0
    if args.params:
        params.update(json.loads(args.params))
    elif not args.no_tune:
        from paper_1910_02639_gb300.autotune import Tuner
        t_tune = time.time()
        tuner = Tuner(dev, ngmax, stream=stream)
        tuner.tune([s])
        params = tuner.params_for([s])[0]
        tune_s = time.time() - t_tune
        del tuner
        torch.cuda.empty_cache()
    cfg.update(bucket_size=params["bucket_size"], beta=params["beta"],
               work_unit=params.get("group_size") or 32,
               find_shape="4 warps, 512-candidate window" if params.get("find_compact")
               else "8 warps, 1024-candidate window",
               pack_leaves=bool(params.get("pack_leaves")),
               tuned=not args.no_tune and not args.params)
    offs = [0, n]

    def step():
        nonlocal tree
        tree = bt.btree_build_batched(x, y, z, h, offs, params, stream=stream, tree=tree)
        bt.btree_find_neighbors_density(tree, m, ngmax, nb, cnt, rho, stream=stream)

    for _ in range(args.warmup):
        step()
    barrier(dist, dev)
    pairs = int(cnt.to(torch.int64).sum().item())
    written = int(torch.clamp(cnt, max=ngmax).to(torch.int64).sum().item())

    # ---- timed region: inputs resident in HBM
    K = args.steps
    f0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    f1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    l0 = bt.btree_kernel_launches()
    barrier(dist, dev)
    t0 = time.time()
    e0.record(stream)
    build_ms = []
    for k in range(K):
        tree = bt.btree_build_batched(x, y, z, h, offs, params, stream=stream, tree=tree)
        build_ms.append(bt.btree_get_info(tree)["build_ms"])
        f0[k].record(stream)
        bt.btree_find_neighbors_density(tree, m, ngmax, nb, cnt, rho, stream=stream)
        f1[k].record(stream)
    e1.record(stream)
    barrier(dist, dev)
    t1 = time.time()
    launches = bt.btree_kernel_launches() - l0
    step_ms = e0.elapsed_time(e1) / K

    # ---- the untuned default: btree_build (s = 16, alpha = beta = 0.5) + find
    dtree = None
    for _ in range(3):
        dtree = bt.btree_build(x, y, z, h, bucket_size=sb, alpha=cfg["alpha"], beta=cfg["beta"],
                               stream=stream, tree=dtree)
        bt.btree_find_neighbors_density(dtree, m, ngmax, nb, cnt, rho, stream=stream)
    barrier(dist, dev)
    e0.record(stream)
    for k in range(K):
        dtree = bt.btree_build(x, y, z, h, bucket_size=sb, alpha=cfg["alpha"], beta=cfg["beta"],
                               stream=stream, tree=dtree)
        bt.btree_find_neighbors_density(dtree, m, ngmax, nb, cnt, rho, stream=stream)
    e1.record(stream)
    barrier(dist, dev)
    default_ms = e0.elapsed_time(e1) / K
    dtree.free()

    # ---- the same step as one CUDA graph (btree_build_find_batched, one set)
    gtree = None
    off = [0, n]
    t_cap = time.perf_counter()
    gtree = bt.btree_build_find_batched(x, y, z, h, off, ngmax, nb, cnt, m=m, rho=rho,
                                        params=params, stream=stream, tree=gtree)
    capture_ms = (time.perf_counter() - t_cap) * 1e3
    for _ in range(2):
        gtree = bt.btree_build_find_batched(x, y, z, h, off, ngmax, nb, cnt, m=m, rho=rho,
                                            params=params, stream=stream, tree=gtree)
    g0 = bt.btree_kernel_launches()
    barrier(dist, dev)
    t0g = time.time()
    e0.record(stream)
    for k in range(K):
        gtree = bt.btree_build_find_batched(x, y, z, h, off, ngmax, nb, cnt, m=m, rho=rho,
                                            params=params, stream=stream, tree=gtree)
    e1.record(stream)
    barrier(dist, dev)
    t1g = time.time()
    graph_launches = bt.btree_kernel_launches() - g0
    graph_ms = e0.elapsed_time(e1) / K
    graph_pairs = int(cnt.to(torch.int64).sum().item())
    gtree.free()
    time.sleep(0.2)
    sampler.stop()
    find_ms = statistics.mean(a.elapsed_time(b) for a, b in zip(f0, f1))
    step_ms_max = reduce_max(dist, step_ms, dev)
    value = pairs * ws / (step_ms_max * 1e-3)

    peak, peak_kind = measured_hbm_peak()
    alg_bytes = n * (16 + 4 + 4 + 4) + 4 * written  # x,y,z,h + m read; count, rho, rows written
    achieved = alg_bytes / (find_ms * 1e-3) / 1e9
    traffic = profiled_traffic(cfg["workload"])
    roofline = {"bound": "hbm", "kernel": "k_find<density> (+k_mass_to_tree)",
                "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic,
                "algorithmic_bytes_per_launch": alg_bytes, "peak_kind": peak_kind}
    insts = profiled_warp_insts(cfg["workload"])
    step_ach = alg_bytes / (step_ms * 1e-3) / 1e9
    step_roofline = {"achieved": round(step_ach, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(step_ach / peak, 4), "note": "same algorithmic bytes over build+find"}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K,
           "warmup": args.warmup, "ms_per_step": step_ms_max, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": cfg, "impl": "gb300",
           "pairs_per_step": pairs, "particles_per_s": n * ws / (step_ms_max * 1e-3),
           "build_ms": round(statistics.mean(build_ms), 4), "find_ms": round(find_ms, 4),
           "roofline": roofline, "step_roofline": step_roofline,
           "gpu_launches": int(launches),
           "tuning_s": round(tune_s, 2),
           "default_params": {"ms_per_step": reduce_max(dist, default_ms, dev),
                              "value": pairs * ws / (reduce_max(dist, default_ms, dev) * 1e-3),
                              "form": "btree_build (s=16, alpha=beta=0.5, 8-warp find) + "
                                      "btree_find_neighbors_density, untuned"},
           "graph_form": {"ms_per_step": reduce_max(dist, graph_ms, dev),
                          "value": graph_pairs * ws / (reduce_max(dist, graph_ms, dev) * 1e-3),
                          "gpu_launches": int(graph_launches), "first_call_ms": round(capture_ms, 3),
                          "identical_pairs": graph_pairs == pairs,
                          "form": "btree_build_find_batched: build+find+density as one CUDA graph "
                                  "launch per step (device-side level and ratio loops)"},
           "clocks": sampler.summary(t0, t1g)}
    if insts:
        # the kernel is instruction-bound: its issue rate against the SMs' peak
        rate = insts / (find_ms * 1e-3)
        pk = issue_peak(out["clocks"].get("sm_mhz"))
        out["issue_roofline"] = {"bound": "issue", "kernel": roofline["kernel"],
                                 "achieved": round(rate / 1e12, 4), "peak": round(pk / 1e12, 4),
                                 "unit": "Twarp-inst/s", "frac": round(rate / pk, 4),
                                 "warp_insts_per_launch": insts,
                                 "note": "instructions from the committed ncu capture (scaled to the "
                                         "workload) over the event-timed launch; peak = 152 SMs x 4 "
                                         "schedulers x SM clock"}

    # ---- end to end through the public API, host buffers (before the batched
    # and serving sections, whose cached device and pinned buffers would
    # otherwise share the box with it)
    if not args.no_e2e:
        torch.cuda.empty_cache()
        out["e2e"] = run_e2e(args, bt, s, cfg, dev, stream, dist, ws, pairs, params)

    # ---- the device's FMA rates: why the distance test filters in FP32
    if rank == 0:
        r = bt.btree_arith_rates(stream)
        out["arith_rates"] = {k: round(v, 1) for k, v in r.items()}
        out["arith_rates"]["fp64_over_fp32"] = round(r["fp64_gflops"] / r["fp32_gflops"], 4)

    # ---- many uneven sets: batched vs the plain per-set path
    if not args.no_batched:
        out["batched"] = run_batched_section(args, bt, dev, stream, dist, rank, ws)

    # ---- serving: Poisson request stream, continuous batching vs plain
    if not args.no_serving:
        out["serving"] = run_serving_section(args, dev, dist, rank, ws)

    # ---- CPU oracle on the host cores (rank 0, N = 1)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(s, cfg, args.cpu_sample)

    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def run_e2e(args, bt, s, cfg, dev, stream, dist, ws, pairs, params):
    """End to end through the public calls, host buffers: every step copies
    the inputs in from pinned host memory, builds, searches with the density,
    packs the rows into compressed rows (only the neighbours travel) and copies
    rows, offsets and densities back to pinned host memory.  The copy-back of
    step k runs on its own stream while step k + 1 computes (two sets of
    output buffers); the timed region ends when the last copy has landed."""
    import torch
    n, g = s.n, cfg["ngmax"]
    hx = [torch.from_numpy(a).pin_memory() for a in (s.x, s.y, s.z, s.h, s.m)]
    dx = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(5)]
    rows = torch.empty(n * g, dtype=torch.int32, device=dev)
    cap = pairs + pairs // 50 + 1024
    cnt = [torch.empty(n, dtype=torch.int32, device=dev) for _ in range(2)]
    rho = [torch.empty(n, dtype=torch.float32, device=dev) for _ in range(2)]
    off = [torch.empty(n + 1, dtype=torch.int64, device=dev) for _ in range(2)]
    csr = [torch.empty(cap, dtype=torch.int32, device=dev) for _ in range(2)]
    h_csr = [torch.empty(cap, dtype=torch.int32).pin_memory() for _ in range(2)]
    h_off = [torch.empty(n + 1, dtype=torch.int64).pin_memory() for _ in range(2)]
    h_rho = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(2)]
    copy_st = torch.cuda.Stream(dev)
    done = [torch.cuda.Event() for _ in range(2)]
    ready = [torch.cuda.Event() for _ in range(2)]
    for e in done:
        e.record(copy_st)
    tree = None
    totals = []

    def step(k):
        nonlocal tree
        b = k & 1
        stream.wait_event(done[b])  # buffer b's previous copy-out has landed
        for d, hsrc in zip(dx, hx):
            d.copy_(hsrc, non_blocking=True)
        tree = bt.btree_build_batched(dx[0], dx[1], dx[2], dx[3], [0, n], params, stream=stream,
                                      tree=tree)
        bt.btree_find_neighbors_density(tree, dx[4], g, rows, cnt[b], rho[b], stream=stream)
        tot = bt.btree_pack_rows(tree, rows, cnt[b], g, off[b], csr[b], stream=stream)
        ready[b].record(stream)
        copy_st.wait_event(ready[b])
        with torch.cuda.stream(copy_st):
            h_csr[b][:tot].copy_(csr[b][:tot], non_blocking=True)
            h_off[b].copy_(off[b], non_blocking=True)
            h_rho[b].copy_(rho[b], non_blocking=True)
        done[b].record(copy_st)
        totals.append(tot)

    for k in range(2):
        step(k)
    torch.cuda.synchronize(dev)
    # this box's device-to-host rate into pinned memory (explains the e2e time)
    nl = min(cap, 1 << 28)
    el0, el1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(copy_st):
        el0.record(copy_st)
        h_csr[0][:nl].copy_(csr[0][:nl], non_blocking=True)
        el1.record(copy_st)
    el1.synchronize()
    d2h_gbs = 4.0 * nl / (el0.elapsed_time(el1) * 1e-3) / 1e9
    K = max(1, min(args.steps, args.e2e_steps))
    totals.clear()
    barrier(dist, dev)
    t0 = time.perf_counter()
    for k in range(K):
        step(k)
    copy_st.synchronize()
    torch.cuda.synchronize(dev)
    ms = (time.perf_counter() - t0) * 1e3 / K
    ms = reduce_max(dist, ms, dev)
    # the host copy of the last step holds every pair exactly once
    ok = int(h_off[(K - 1) & 1][n].item()) == pairs
    tot = statistics.mean(totals)
    return {"value": pairs * ws / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": K,
            "h2d_bytes_per_step": 5 * 4 * n,
            "d2h_bytes_per_step": int(4 * tot + 8 * (n + 1) + 4 * n),
            "result": "compressed rows (every neighbour, ascending) + offsets + densities",
            "overlap": "copy-back of step k overlaps step k+1 (two output buffers)",
            "d2h_gbs_measured": round(d2h_gbs, 1),
            "complete": bool(ok)}


# ---------------------------------------------------------------- batched sets
def _timed(fn, stream, steps, warmup=3):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / steps


def _batched_by_kind(bt, sets, kinds, tuner, dev, stream, ngmax, K):
    """The tuned batched build + search of each kind of set alone (this
    rank's sets), with the build and the search timed apart."""
    import torch
    from paper_1910_02639_gb300.batch import DeviceSets
    out = {}
    for kind in sorted(set(kinds)):
        sub = [s for s, k in zip(sets, kinds) if k == kind]
        ds = DeviceSets(sub, dev, ngmax)
        p = tuner.params_for(sub)
        ms = _timed(lambda: ds.run_batched(p, stream), stream, K)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        bms = fms = 0.0
        for _ in range(K):
            ev[0].record(stream)
            ds._tree = bt.btree_build_batched(ds.x, ds.y, ds.z, ds.h, ds.offsets, ds.params_list(p),
                                              stream=stream, tree=ds._tree)
            ev[1].record(stream)
            bt.btree_find_neighbors_density(ds._tree, ds.m, ds.ngmax, ds.nb, ds.cnt, ds.rho, stream=stream)
            ev[2].record(stream)
            ev[2].synchronize()
            bms += ev[0].elapsed_time(ev[1]) / K
            fms += ev[1].elapsed_time(ev[2]) / K
        pairs = int(ds.cnt.to(torch.int64).sum().item())
        out[kind] = {"sets": len(sub), "particles": int(sum(s.n for s in sub)), "pairs": pairs,
                     "ms_per_step": ms, "pairs_per_s": pairs / (ms * 1e-3),
                     "build_ms": bms, "find_ms": fms,
                     "max_count": int(ds.cnt.max().item()) if sub else 0}
        ds.free()
        del ds
    torch.cuda.empty_cache()
    return out


def run_batched_section(args, bt, dev, stream, dist, rank, ws):
    """256 independent sets, sizes log-uniform in [1e3, 1e6] (uniform cube,
    1/r sphere, Plummer; 50-150 target neighbours), ngmax 256.  Each rank
    takes a size-balanced share of the sets (no collective on the data path).
    Three forms on the same sets, same outputs: the plain path (build + find
    per set), one batched call with the default parameters, one batched call
    with the autotuner's per-size-class parameters."""
    import torch
    from paper_1910_02639_gb300 import workloads as wl
    from paper_1910_02639_gb300.autotune import Tuner
    from paper_1910_02639_gb300.batch import DeviceSets, list_checksum, shard_sets
    specs = wl.batched_specs(args.batched_sets, seed=1914)
    mine = shard_sets([sp[1] for sp in specs], ws)[rank]
    sets = [wl.make_set(*specs[i]) for i in mine]
    ngmax = 256
    ds = DeviceSets(sets, dev, ngmax)
    K = args.batched_steps
    t0 = time.time()
    tuner = Tuner(dev, ngmax, stream=stream)
    tuner.tune(sets)
    tune_s = time.time() - t0
    tuned = tuner.params_for(sets)

    plain_ms = _timed(lambda: ds.run_plain(None, stream), stream, K)
    ref = (int(ds.cnt.to(torch.int64).sum().item()), list_checksum(ds.nb, ds.cnt, ngmax))
    rho_ref = ds.rho.clone()
    l0 = bt.btree_kernel_launches()
    batched_ms = _timed(lambda: ds.run_batched(None, stream), stream, K)
    launches_batched = (bt.btree_kernel_launches() - l0) // (K + 3)
    same_b = ((int(ds.cnt.to(torch.int64).sum().item()), list_checksum(ds.nb, ds.cnt, ngmax)) == ref
              and torch.equal(ds.rho, rho_ref))
    tuned_ms = _timed(lambda: ds.run_batched(tuned, stream), stream, K)
    same_t = ((int(ds.cnt.to(torch.int64).sum().item()), list_checksum(ds.nb, ds.cnt, ngmax)) == ref
              and torch.equal(ds.rho, rho_ref))
    l0 = bt.btree_kernel_launches()
    graph_ms = _timed(lambda: ds.run_graph(tuned, stream), stream, K)
    launches_graph = (bt.btree_kernel_launches() - l0) // (K + 3)
    same_g = ((int(ds.cnt.to(torch.int64).sum().item()), list_checksum(ds.nb, ds.cnt, ngmax)) == ref
              and torch.equal(ds.rho, rho_ref))
    pairs = ref[0]
    all_pairs = pairs
    if dist:
        t = torch.tensor([pairs], dtype=torch.float64, device=dev)
        dist.all_reduce(t)
        all_pairs = int(t.item())
    plain_ms, batched_ms, tuned_ms, graph_ms = (reduce_max(dist, v, dev)
                                                for v in (plain_ms, batched_ms, tuned_ms, graph_ms))
    ds.free()
    del ds
    by_kind = _batched_by_kind(bt, sets, [specs[i][0] for i in mine], tuner, dev, stream, ngmax, K)
    rate = lambda ms: all_pairs / (ms * 1e-3)
    table = {"%d,%d" % k: {kk: v.get(kk) for kk in ("bucket_size", "beta", "group_size", "find_compact",
                                                    "pack_leaves")}
             for k, v in tuner.table.items()}
    return {"workload": f"batched_{args.batched_sets}_sets", "n": int(sum(sp[1] for sp in specs)),
            "nsets": len(specs), "ngmax": ngmax, "scaling": "strong", "sets_per_rank": len(mine),
            "pairs_per_step": all_pairs, "unit": UNIT,
            "plain": {"value": rate(plain_ms), "ms_per_step": plain_ms,
                      "form": "btree_build + fused find per set, s=16, beta=0.5"},
            "batched": {"value": rate(batched_ms), "ms_per_step": batched_ms,
                        "launches_per_step": int(launches_batched),
                        "form": "btree_build_batched + one fused find, s=16, beta=0.5",
                        "identical_to_plain": bool(same_b)},
            "tuned": {"value": rate(tuned_ms), "ms_per_step": tuned_ms,
                      "identical_to_plain": bool(same_t), "table": table,
                      "tuning_s": round(tune_s, 2), "trials": tuner.trials},
            "graph": {"value": rate(graph_ms), "ms_per_step": graph_ms,
                      "launches_per_step": int(launches_graph),
                      "form": "btree_build_find_batched with the tuned parameters: one CUDA graph "
                              "launch per step, level and ratio loops as device-side while-nodes",
                      "identical_to_plain": bool(same_g)},
            "by_kind": by_kind,
            "speedup_batched_vs_plain": plain_ms / batched_ms,
            "speedup_graph_vs_plain": plain_ms / graph_ms,
            "speedup_tuned_vs_plain": plain_ms / tuned_ms,
            "steps": K, "warmup": 3}


# ---------------------------------------------------------------- serving
def run_serving_section(args, dev, dist, rank, ws):
    """Poisson arrivals (200 requests/s), sizes log-uniform in [1e4, 2e6], the
    three distributions of the batched workload; each request = copy in +
    build + find + density, results left in HBM.  Served by the
    continuous-batching loop (4 slots) and, under the same arrivals, by the
    plain path one job at a time.  Then the same requests all at once
    (saturated) for throughput.  Each rank serves its own share of the
    stream.  Unless --no-tune, every request carries the autotuner's
    parameters for its class of set (size, spread of h); the plain path uses
    the tree parameters among them."""
    import numpy as np
    import torch
    from paper_1910_02639_gb300 import serving
    from paper_1910_02639_gb300 import workloads as wl
    from paper_1910_02639_gb300.batch import list_checksum, shard_sets
    specs = wl.request_stream(args.serving_requests, seed=1915, rate=200.0)
    mine = shard_sets([1] * len(specs), ws)[rank]  # round-robin by arrival
    ngmax = 256
    sets = [wl.make_set(*specs[i][1:]) for i in mine]
    reqs = [serving.make_request(i, specs[i][0], s) for i, s in zip(mine, sets)]
    tuned = not args.no_tune
    if tuned:
        # the autotuner's parameters per class of set, for every request (the
        # plain path takes the tree parameters among them: s, alpha, beta)
        from paper_1910_02639_gb300.autotune import Tuner
        tuner = Tuner(dev, ngmax)
        tuner.tune(sets)
        for r, p in zip(reqs, tuner.params_for(sets)):
            r.params = p
        del tuner
        torch.cuda.empty_cache()
    del sets
    sums, pairs = {}, {}

    def grab(tag):
        def f(res):
            if res.error is not None:
                raise RuntimeError(f"request {res.rid} failed: {res.error}")
            c = int(res.cnt.to(torch.int64).sum().item())
            rb = int(res.rho.view(torch.int32).to(torch.int64).sum().item())
            sums[(tag, res.rid)] = (c, list_checksum(res.nb, res.cnt, ngmax), rb)
            pairs[res.rid] = c
        return f

    # warm-up (kernels, allocator, trees)
    srv = serving.Server(dev, ngmax=ngmax, slots=args.serving_slots)
    try:
        serving.replay(srv, [serving.make_request(-1, 0.0, wl.make_set("uniform_cube", 50_000, 1, 100.0))])
        served = serving.replay(srv, reqs)
        for r in reqs:
            r.arrival = 0.0
        sat = serving.replay(srv, reqs)
        # the results checked outside the timed replays (the checks run in
        # the client loop and would delay the submissions)
        serving.replay(srv, reqs, on_result=grab("served"))
    finally:
        srv.close()
    for r, sp in zip(reqs, (specs[i] for i in mine)):
        r.arrival = sp[0]
    serving.replay_plain([serving.make_request(-1, 0.0, wl.make_set("uniform_cube", 50_000, 1, 100.0))],
                         dev, ngmax)
    plain = serving.replay_plain(reqs, dev, ngmax)
    for r in reqs:
        r.arrival = 0.0
    plain_sat = serving.replay_plain(reqs, dev, ngmax)
    serving.replay_plain(reqs, dev, ngmax, on_result=grab("plain"))
    total = sum(pairs.values())
    same = all(sums[("served", r.rid)] == sums[("plain", r.rid)] for r in reqs)
    st = serving.latency_stats(served, total)
    sp_ = serving.latency_stats(plain, total)
    st_sat = serving.latency_stats(sat, total)["pairs_per_s"]
    sp_sat = serving.latency_stats(plain_sat, total)["pairs_per_s"]
    if dist:
        # each rank served its own share of the stream: throughputs add up;
        # latency percentiles are rank 0's
        t = torch.tensor([st["pairs_per_s"], sp_["pairs_per_s"], st_sat, sp_sat, float(same == 0)],
                         dtype=torch.float64, device=dev)
        dist.all_reduce(t)
        st["pairs_per_s"], sp_["pairs_per_s"], st_sat, sp_sat = (float(v) for v in t[:4])
        same = t[4].item() == 0.0
    sweep = run_serving_sweep(args, dev, reqs, pairs, ngmax) if not args.no_serving_sweep else None
    out = {"workload": f"poisson_{args.serving_requests}_requests_200_per_s",
           "requests": len(reqs), "particles": int(sum(r.n for r in reqs)), "pairs": total,
           "slots": args.serving_slots, "ngmax": ngmax,
           "params": "autotuned per class of set (the plain path: s, alpha, beta)" if tuned
                     else "defaults (s = 16, alpha = beta = 0.5)",
           "served": {k: st[k] for k in ("p50_ms", "p99_ms", "mean_ms", "pairs_per_s")},
           "plain": {k: sp_[k] for k in ("p50_ms", "p99_ms", "mean_ms", "pairs_per_s")},
           "saturated_pairs_per_s": {"served": st_sat, "plain": sp_sat},
           "ranks": ws,
           "mean_batch_size": float(np.mean([r.batch_size for r in served])),
           "identical_to_plain": bool(same)}
    if sweep is not None:
        out["sweep"] = sweep
    return out


def run_serving_sweep(args, dev, pool, pool_pairs, ngmax):
    """Arrival-rate sweep: for each rate, args.serving_sweep_requests Poisson
    arrivals (seeded) whose sets are drawn in turn from the request pool of
    the 200-request stream (same pinned host arrays, same per-class
    parameters); served by the continuous-batching loop and by the plain path
    under the same arrivals.  Reports latency percentiles, throughput and how
    many requests a batch held."""
    import numpy as np
    from paper_1910_02639_gb300 import serving
    out = []
    nreq = args.serving_sweep_requests
    for k, rate in enumerate(args.serving_rates):
        rng = np.random.Generator(np.random.PCG64(1917 + k))
        t = np.cumsum(rng.exponential(1.0 / rate, nreq))
        reqs = []
        for i in range(nreq):
            src = pool[i % len(pool)]
            r = serving.Request(i, float(t[i]), src.x, src.y, src.z, src.h, src.m, dict(src.params))
            reqs.append(r)
        total = sum(pool_pairs[pool[i % len(pool)].rid] for i in range(nreq))
        srv = serving.Server(dev, ngmax=ngmax, slots=args.serving_slots)
        try:
            served = serving.replay(srv, reqs)
            tl = list(srv.timeline)
        finally:
            srv.close()
        plain = serving.replay_plain(reqs, dev, ngmax)
        st = serving.latency_stats(served, total)
        sp_ = serving.latency_stats(plain, total)
        # device time covered by two or more slots at once
        ev = sorted([(a, 1) for _, _, a, _, _ in tl] + [(b, -1) for _, _, _, b, _ in tl])
        depth, last, multi, busy = 0, None, 0.0, 0.0
        for x, d in ev:
            if last is not None and depth > 0:
                busy += x - last
                if depth > 1:
                    multi += x - last
            depth += d
            last = x
        out.append({"rate_per_s": rate, "requests": nreq, "pairs": total,
                    "served": {kk: st[kk] for kk in ("p50_ms", "p99_ms", "mean_ms", "pairs_per_s")},
                    "plain": {kk: sp_[kk] for kk in ("p50_ms", "p99_ms", "mean_ms", "pairs_per_s")},
                    "mean_batch_size": float(np.mean([r.batch_size for r in served])),
                    "max_batch_size": int(max(r.batch_size for r in served)),
                    "batches": len(tl),
                    "device_overlap_frac": multi / busy if busy > 0 else 0.0})
    return out


# ---------------------------------------------------------------- CPU oracle
def cpu_baseline(s, cfg, sample):
    """The oracle as it stands: BuildTree over the whole set, FindNeighbors for
    a contiguous sample of queries; the build time is charged pro rata."""
    import numpy as np
    import oracle
    oracle.build()
    n = s.n
    q = min(sample, n)
    q0 = (n - q) // 2
    t0 = time.perf_counter()
    tr = oracle.OracleTree(s.x, s.y, s.z, bucket_size=cfg["bucket_size"], alpha=cfg["alpha"],
                           beta=cfg["beta"])
    t1 = time.perf_counter()
    _, c = tr.find(s.h, cfg["ngmax"], q0, q0 + q)
    t2 = time.perf_counter()
    pairs = int(np.asarray(c, dtype=np.int64).sum())
    secs = (t1 - t0) * q / n + (t2 - t1)
    # the brute-force definition on the small uniform configuration (32768
    # particles, every query against every particle), for scale
    from paper_1910_02639_gb300 import workloads as wl
    u = wl.uniform_cube(32768, seed=1911)
    t3 = time.perf_counter()
    _, cb = oracle.find_brute(u.x, u.y, u.z, u.h, 256)
    t4 = time.perf_counter()
    pb = int(np.asarray(cb, dtype=np.int64).sum())
    return {"value": pairs / secs, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"BuildTree on all {n} particles ({t1 - t0:.2f} s, charged pro rata) + "
                      f"FindNeighbors for particles [{q0}, {q0 + q}) ({t2 - t1:.2f} s), {pairs} pairs",
            "build_s": round(t1 - t0, 3), "find_s": round(t2 - t1, 3),
            "brute_force_uniform_32768": {"pairs_per_s": pb / (t4 - t3), "s": round(t4 - t3, 3),
                                          "pairs": pb}}


def run_reference(args):
    """The reference arm: the CPU oracle on the host cores, on the same
    workload and metric; each step a bounded sample."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import oracle
    oracle.build()
    s, cfg = make_workload(args.workload)
    n = s.n
    q = min(args.ref_sample, n)
    times, pairs_l = [], []
    for k in range(args.warmup + args.steps):
        q0 = (k * q) % max(n - q, 1)
        t0 = time.perf_counter()
        tr = oracle.OracleTree(s.x, s.y, s.z, bucket_size=cfg["bucket_size"], alpha=cfg["alpha"],
                               beta=cfg["beta"])
        t1 = time.perf_counter()
        _, c = tr.find(s.h, cfg["ngmax"], q0, q0 + q)
        t2 = time.perf_counter()
        del tr
        if k >= args.warmup:
            times.append((t1 - t0) * q / n + (t2 - t1))
            pairs_l.append(int(np.asarray(c, dtype=np.int64).sum()))
    value = sum(pairs_l) / sum(times)
    cores = oracle.num_threads()
    sample = (f"per step: oracle BuildTree on all {n} particles (charged pro rata {q}/{n}) + "
              f"FindNeighbors for {q} consecutive particles")
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": cfg, "impl": "reference",
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="slab1e7")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=1_000_000)
    ap.add_argument("--ref-sample", type=int, default=200_000)
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--params", default="",
                    help='fixed set parameters as JSON (no tuning), e.g. {"find_compact": true}')
    ap.add_argument("--batched-sets", type=int, default=256)
    ap.add_argument("--batched-steps", type=int, default=5)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=200)
    ap.add_argument("--serving-slots", type=int, default=4)
    ap.add_argument("--no-serving-sweep", action="store_true")
    ap.add_argument("--serving-sweep-requests", type=int, default=2000)
    ap.add_argument("--serving-rates", type=float, nargs="+", default=[200.0, 1000.0, 4000.0])
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
