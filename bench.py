#!/usr/bin/env python
"""Near-field correction points/sec on GB300: one step = build_near_lists +
gen_corrections (geometry, near lists, far order q_j, smooth/annulus moments, adaptive
near moments, self weights, V contraction into the CSR) over the whole surface.

Default workload: CFIE D - ik S, k = 2 pi, ellipsoid with semi-axes (1, 2, 3) as 1280
degree-6 patches (28 nodes each, 35,840 points), eps = 1e-9, FP64; all nodes are
targets.  Metric: N / T_step (the paper's S_init = N / T_init).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain FP64 restatement in oracle/) on the
host cores, each step a bounded sample of the same workload.  Under torchrun every
rank runs an independent copy of the workload (weak scaling, no collective on the data
path); rank 0 prints one JSON line.
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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("near-field correction points/sec on 1 GB300 (FP64 vs mixed/batched) at "
          "ε=1e-6/1e-9")
UNIT = "points/s"
WORKLOAD = "CFIE D-ikS k=2pi ellipsoid(1,2,3) 1280 order-6 patches (35,840 pts) eps=1e-9 FP64"


def workload_name(patches, points, eps, precision="fp64"):
    """WORKLOAD for the default configuration, else the same description at other sizes."""
    if patches == 1280 and eps == 1e-9 and precision == "fp64":
        return WORKLOAD
    form = "FP64" if precision == "fp64" else "mixed"
    return (f"CFIE D-ikS k=2pi ellipsoid(1,2,3) {patches} order-6 patches ({points:,} pts) "
            f"eps={eps:g} {form}")

# Algorithmic FLOPs of one (target, leaf node) evaluation in the adaptive kernel: the
# kernel value (difference, r^2, phase, e^{ikr}/(4 pi r), S and D parts, CFIE combination:
# 20 arithmetic operations, and sqrt, reciprocal and sincos counted as one each), plus the
# contraction onto n Koornwinder moments (complex x real: 4 per moment).
KERNEL_FLOPS = 20 + 3


def flops_per_eval(n):
    return KERNEL_FLOPS + 4 * n


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batched-scale", type=float, default=1.0,
                    help="patch-count scale of the 64-torus batch variant (0: skip it; 1: the "
                         "full batch)")
    ap.add_argument("--no-table1", action="store_true",
                    help="skip the twisted-torus sweep over order p and eps (the paper's Table 1)")
    ap.add_argument("--no-table2", action="store_true",
                    help="skip the twisted-torus sweep over the patches' aspect ratio (the "
                         "paper's Table 2: p = 4, eps = 5e-7, five grids)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the 40,000-patch torus (k=20, eps=1e-9; FP64 and mixed, and the "
                         "direct-sum apply on a 100,000-point subset)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--s", "--subdiv", dest="s", type=int, default=8,
                    help="icosahedral refinement (1280 patches at 8); under torchrun spell it "
                         "--subdiv (the launcher takes --s for one of its own options)")
    ap.add_argument("--leaf-order", type=int, default=0,
                    help="smooth rule used on subtriangles (0: the patch's far order q_j)")
    ap.add_argument("--eps", type=float, default=1e-9)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="form of the timed steps (the variants compare both)")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the mixed-precision and eps=1e-6 comparison runs")
    return ap.parse_args()


# ----------------------------------------------------------------------------- oracle leg
def _oracle_worker(job):
    """Oracle corrections for some patches of the workload (runs in a spawned process)."""
    import numpy as np  # noqa: F401
    s_div, patches, dirs_seed, eps, leaf = job
    from oracle import corrections as C
    from oracle import geometry
    from paper_2006_02545_gb300 import workloads as W
    wl = W.ellipsoid_cfie_k2pi(s_div)
    surf = wl.surface
    pts = geometry.make_patches(surf.deg, surf.node_off, surf.xyz)
    p = C.Params(eps=eps, eta=wl.eta, test_dirs=W.test_directions(dirs_seed), leaf_order=leaf)
    t0 = time.perf_counter()
    C.gen_corrections(surf.deg, surf.node_off, surf.xyz, wl.tgt_xyz, wl.tgt_node, wl.kernel, wl.k,
                      wl.alpha, wl.beta, params=p, patches=pts, only_patches=patches)
    return len(patches), time.perf_counter() - t0


def oracle_sample(s_div, n_patches_total, workers, per_worker, seed, pool, eps=1e-9, leaf=0):
    """Time the oracle on workers*per_worker patches spread over the surface.
    Throughput = points of the sampled patches / the slowest worker's compute time."""
    n = 28
    total = workers * per_worker
    stride = max(1, n_patches_total // total)
    picks = [(i * stride + seed) % n_patches_total for i in range(total)]
    jobs = [(s_div, picks[w::workers], 7, eps, leaf) for w in range(workers)]
    res = pool.map(_oracle_worker, jobs)
    done = sum(r[0] for r in res)
    worst = max(r[1] for r in res)
    return done * n / worst, done, worst


def make_pool(workers):
    import multiprocessing as mp
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    return mp.get_context("spawn").Pool(workers)


def run_reference(args, rank):
    if rank != 0:
        return
    workers = max(1, min(16, os.cpu_count() or 1))
    pool = make_pool(workers)
    npat = 20 * args.s * args.s
    vals, times = [], []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        v, done, worst = oracle_sample(args.s, npat, workers, 1, it * 37, pool, args.eps,
                                       args.leaf_order)
        if it >= args.warmup:
            vals.append(v)
            times.append(time.perf_counter() - t0)
    pool.close()
    value = statistics.median(vals)
    sample = (f"{workers} patches per step (1 per worker) of {npat}; throughput = sampled "
              f"points / slowest worker's compute time")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(npat, 28 * npat, args.eps), "patches": npat,
                   "order": 6, "precision": "fp64", "points": 28 * npat, "eps": args.eps,
                   "leaf_order": args.leaf_order or "q_j",
                   "l2": "host cores: no device cache to flush",
                   "tuning": "none (the oracle has no tuner)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" +
                                       self.FIELDS, "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.strip().split(",") for r in self.f.read().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = max(mx, float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------- our leg
TUNING_GENERATIONS = 6
# arithmetic of the pair evaluations by form (lcq_counters [7]); FP64 everywhere else
MIXED_DTYPE = {"fp64": "f64", "fp32": "f32+f64", "two-float": "f32x2+f64",
               "fp32+two-float": "f32+f32x2+f64"}
FORM_NAMES = {0: "fp64", 1: "fp32", 2: "two-float", 3: "fp32+two-float"}  # lcq_counters [7]
KERNEL_SOURCES = ("lcq_common.cuh", "lcq_device.cuh", "lcq_tc.cuh")  # k_adaptive and its helpers


def kernel_source_sha():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2006_02545_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def traffic_for(kernel_name):
    """DRAM bytes per launch of `kernel_name` from the committed ncu summary, if it was
    taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(kernel_name)
        sha = kernel_source_sha()
        if rec and rec.get("src_sha256") == sha:
            return rec.get("bytes_per_launch")
    except (OSError, ValueError):
        pass
    return None


def table2_sweep(ctx, lcq, W, dev, stream, flush):
    """The paper's Table 2 on its twisted torus: p = 4 (degree 3), S, k = 1, eps = 5e-7 on the
    five grids of the aspect-ratio sweep; per column the patch count, the average aspect
    ratio, alpha = N_over / N, m = nnz / N and S_init = N / T_init (the last of the tuner's
    generations, one warm-up and one timed)."""
    import torch
    rows = []
    for col, (n_u, n_v) in enumerate(W.TABLE2_GRIDS, start=1):
        ts = W.stellarator(n_u, n_v, 3)
        tx, ttn = W.onsurface_targets(ts)
        tds = lcq.DeviceSurface(ts.deg, ts.node_off, torch.from_numpy(ts.xyz).to(dev))
        tx_d = torch.from_numpy(tx).to(dev)
        ttn_d = torch.from_numpy(ttn).to(dev)
        tp = lcq.params(5e-7, test_dirs=W.test_directions(7))
        ms = []
        for _ in range(TUNING_GENERATIONS + 2):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            near = lcq.build_near_lists(ctx, tds, tx_d, ttn_d, tp)
            corr = lcq.gen_corrections(ctx, tds, near, "S", 1.0, tp)
            e1.record(stream)
            st = ctx.sync()
            ms.append(e0.elapsed_time(e1))
            t_stages = ctx.stage_times()[0]
            nnz, n_over = corr.info()
            corr.close()
            near.close()
        rows.append({"column": col, "grid": [n_u, n_v], "patches": ts.n_patches,
                     "points": ts.n_points, "a_avg": float(W.aspect_ratios(ts).mean()),
                     "alpha": n_over / ts.n_points, "m": nnz / ts.n_points,
                     "S_init": ts.n_points / (ms[-1] / 1e3), "status": st,
                     "stages_ms": [round(float(x), 3) for x in t_stages]})
        del tds, tx_d, ttn_d
    return rows


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2006_02545_gb300 import build as B
    B.build()
    from paper_2006_02545_gb300 import lcq
    from paper_2006_02545_gb300 import workloads as W
    from paper_2006_02545_gb300.replicas import job_throughput, max_over_ranks

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    wl = W.ellipsoid_cfie_k2pi(args.s)
    surf = wl.surface
    N, NT, P = surf.n_points, wl.tgt_xyz.shape[1], surf.n_patches
    n = 28
    ctx = lcq.Context(local_rank)
    stream = ctx.stream
    peaks = lcq.pipe_peaks(local_rank)   # measured denominators of the roofline fractions
    xyz_d = torch.from_numpy(surf.xyz).to(dev)
    tx_d = torch.from_numpy(np.ascontiguousarray(wl.tgt_xyz)).to(dev)
    tn_d = torch.from_numpy(wl.tgt_node).to(dev)
    ds = lcq.DeviceSurface(surf.deg, surf.node_off, xyz_d)
    prm = lcq.params(args.eps, eta=wl.eta, test_dirs=W.test_directions(7),
                     leaf_order=args.leaf_order)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        near = lcq.build_near_lists(ctx, ds, tx_d, tn_d, prm)
        corr = lcq.gen_corrections(ctx, ds, near, wl.kernel, wl.k, prm, wl.alpha, wl.beta,
                                   precision=args.precision)
        return near, corr

    # the context's group-size tuner times one candidate per generation on a new workload
    # (at most five here): untimed generations before the warm-up settle it, so that the
    # timed steps run its choice whatever W is
    for _ in range(TUNING_GENERATIONS + args.warmup):
        near, corr = step()
        st = ctx.sync()
        corr.close()
        near.close()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local_rank) if rank == 0 else None
    step_ms, adapt_ms, stages, statuses, launches, nodes = [], [], [], [], 0, 0
    tree_nodes = tests = group_size = items = main_forms = 0
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        near, corr = step()
        e1.record(stream)
        st = ctx.sync()
        statuses.append(st)
        step_ms.append(e0.elapsed_time(e1))
        ms, nl = ctx.stage_times()
        stages.append(ms)
        adapt_ms.append(ms[3])
        launches += nl
        cnt = ctx.counters()
        nodes = int(cnt[1])
        tree_nodes = int(cnt[4])
        tests = int(cnt[0])
        group_size, items = int(cnt[5]), int(cnt[6])
        main_forms = int(cnt[7])
        corr.close()
        near.close()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop() if clocks else None
    total_ms = max_over_ranks(sum(step_ms), dev)
    value = job_throughput(N, args.steps, world, total_ms)

    # FP64 vs mixed at eps = 1e-9 and 1e-6: throughput and the applied potential's
    # relative L2 difference from the FP64 result on the same density
    variants = None
    if not args.no_variants:
        variants = {}
        sig = torch.from_numpy(W.density(N, 0)).to(dev)
        ref_u = {}
        for eps in (args.eps, 1e-6):
            for prec in ("fp64", "mixed"):
                p2 = lcq.params(eps, eta=wl.eta, test_dirs=W.test_directions(7),
                                leaf_order=args.leaf_order)
                times, ad = [], []
                # the first generations of a new (precision, tolerance) key time the group
                # size tuner's candidates (at most five); the last two are timed
                nit = 7
                for it in range(nit):
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    near = lcq.build_near_lists(ctx, ds, tx_d, tn_d, p2)
                    corr = lcq.gen_corrections(ctx, ds, near, wl.kernel, wl.k, p2, wl.alpha, wl.beta,
                                               precision=prec)
                    e1.record(stream)
                    st = ctx.sync()
                    if it >= nit - 2:
                        times.append(e0.elapsed_time(e1))
                        ad.append(ctx.stage_times()[0][3])
                    if it < nit - 1:
                        corr.close()
                        near.close()
                forms = int(ctx.counters()[7])
                u = lcq.apply_corrected_CFIE(ctx, ds, near, corr, sig, NT).cpu().numpy()
                val = corr.export(NT)[2].copy()
                corr.close()
                near.close()
                key = f"{prec}_eps{eps:g}"
                rec = {"value": N / (statistics.mean(times) / 1e3), "unit": UNIT,
                       "ms_per_step": statistics.mean(times), "adaptive_ms": statistics.mean(ad),
                       "status": st}
                if prec == "fp64":
                    ref_u[eps] = (u, val)
                else:
                    ru, rv = ref_u[eps]
                    rec["rel_l2_vs_fp64"] = float(np.linalg.norm(u - ru) / np.linalg.norm(ru))
                    rec["csr_rel_l2_vs_fp64"] = float(np.linalg.norm(val - rv) / np.linalg.norm(rv))
                    rec["fp32_used"] = forms != 0
                    rec["pair_form"] = FORM_NAMES[forms]
                variants[key] = rec

    # the 20-patch sphere (single layer, k = 1, eps = 1e-6, eta = 1.25): 300 points, a
    # latency-bound case (about 50 launches and three host synchronizations per step)
    small = None
    if not args.no_variants:
        sw = W.sphere_s_k1()
        sds = lcq.DeviceSurface(sw.surface.deg, sw.surface.node_off,
                                torch.from_numpy(sw.surface.xyz).to(dev))
        sx = torch.from_numpy(sw.tgt_xyz).to(dev)
        stn = torch.from_numpy(sw.tgt_node).to(dev)
        sp = lcq.params(sw.eps, eta=sw.eta, test_dirs=W.test_directions(7))
        times, sst = [], []
        for it in range(16):   # the first generations time the group-size candidates
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            near = lcq.build_near_lists(ctx, sds, sx, stn, sp)
            corr = lcq.gen_corrections(ctx, sds, near, "S", 1.0, sp)
            e1.record(stream)
            st_s = ctx.sync()
            if it >= 8:
                times.append(e0.elapsed_time(e1))
                sst.append(ctx.stage_times()[0])
                s_group = int(ctx.counters()[5])
            corr.close()
            near.close()
        # the same generation captured once as a CUDA graph (lcq_plan) and replayed: the
        # geometry refresh and stages 1-6 with no host synchronization (near lists frozen)
        near = lcq.build_near_lists(ctx, sds, sx, stn, sp)
        corr = lcq.gen_corrections(ctx, sds, near, "S", 1.0, sp)
        ctx.sync()
        plan = lcq.Plan(ctx, sds, near, corr)
        gtimes = []
        for it in range(13):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.launch()
            e1.record(stream)
            st_g = ctx.sync()
            if it >= 3:
                gtimes.append(e0.elapsed_time(e1))
        g_launches = int(ctx.stage_times()[1])
        plan.close()
        corr.close()
        near.close()
        small = {"workload": sw.name, "points": sw.surface.n_points,
                 "value": sw.surface.n_points / (statistics.median(times) / 1e3), "unit": UNIT,
                 "ms_per_step": statistics.median(times), "status": st_s,
                 "group_size": s_group,
                 "graph": {"ms_per_step": statistics.median(gtimes),
                           "value": sw.surface.n_points / (statistics.median(gtimes) / 1e3),
                           "unit": UNIT, "status": st_g, "launches_per_step": g_launches,
                           "note": "lcq_plan replay: geometry refresh + generation, near "
                                   "lists frozen, no host synchronization"},
                 "stages_ms": dict(zip(["near_lists", "far_order", "smooth_annulus", "adaptive",
                                        "self", "v2c"],
                                       [statistics.median(x[i] for x in sst) for i in range(6)]))}

    # 64 independent tori in one batched generation against the same surfaces one by one
    batched = None
    if not args.no_variants and args.batched_scale > 0:
        bs, poff, phys, _ = W.batched_tori_batch(64, 0, args.batched_scale)
        bx, btn = W.onsurface_targets(bs)
        bds = lcq.DeviceSurface(bs.deg, bs.node_off, torch.from_numpy(bs.xyz).to(dev))
        bx_d = torch.from_numpy(bx).to(dev)
        btn_d = torch.from_numpy(btn).to(dev)
        bp = lcq.params(1e-6, test_dirs=W.test_directions(7))
        # warm every degree's kernels on a small batch, then time one full generation
        ws_, wpoff = W.concat_surfaces([W.torus(6, 12, d) for d in range(3, 9)],
                                       [(8.0 * i, 0.0, 0.0) for i in range(6)])
        wphys = [(5.0, 1.0, -5j, 1e-6)] * 6
        wds = lcq.DeviceSurface(ws_.deg, ws_.node_off, torch.from_numpy(ws_.xyz).to(dev))
        wx, wtn = W.onsurface_targets(ws_)
        wnear = lcq.build_near_lists_batched(ctx, wds, wpoff, torch.from_numpy(wx).to(dev),
                                             torch.from_numpy(wtn).to(dev), lcq.params(1e-6))
        lcq.gen_corrections_batched(ctx, wds, wnear, "CFIE", wphys, lcq.params(1e-6)).close()
        ctx.sync()
        wnear.close()
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        near = lcq.build_near_lists_batched(ctx, bds, poff, bx_d, btn_d, bp)
        corr = lcq.gen_corrections_batched(ctx, bds, near, "CFIE", phys, bp)
        e1.record(stream)
        st_b = ctx.sync()
        times = [e0.elapsed_time(e1)]
        b_launches = ctx.stage_times()[1]
        corr.close()
        near.close()
        # the same batch in the mixed form (per surface: FP32 pairs at eps = 1e-6,
        # two-float ones at 1e-9)
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        near = lcq.build_near_lists_batched(ctx, bds, poff, bx_d, btn_d, bp)
        corr = lcq.gen_corrections_batched(ctx, bds, near, "CFIE", phys, bp, precision="mixed")
        e1.record(stream)
        st_bm = ctx.sync()
        bm_ms = e0.elapsed_time(e1)
        bm_forms = int(ctx.counters()[7])
        corr.close()
        near.close()
        one_ms, one_launches = 0.0, 0
        for i, (k, a, b, eps) in enumerate(phys):
            n0, n1 = int(bs.node_off[poff[i]]), int(bs.node_off[poff[i + 1]])
            dsi = lcq.DeviceSurface(bs.deg[poff[i]:poff[i + 1]],
                                    bs.node_off[poff[i]:poff[i + 1] + 1] - n0, bds.xyz[:, n0:n1].contiguous())
            xi = bx_d[:, n0:n1].contiguous()
            ti = btn_d[n0:n1] - n0
            pi = lcq.params(eps, test_dirs=W.test_directions(7))
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            near = lcq.build_near_lists(ctx, dsi, xi, ti, pi)
            corr = lcq.gen_corrections(ctx, dsi, near, "CFIE", k, pi, a, b)
            e1.record(stream)
            ctx.sync()
            one_ms += e0.elapsed_time(e1)
            one_launches += ctx.stage_times()[1]
            corr.close()
            near.close()
        bms = statistics.mean(times)
        batched = {"workload": f"64 perturbed tori (R=2, r=1), patch counts U[200,5000] x "
                               f"{args.batched_scale:g}, degree U{{3..8}}, k U[1,20], eps "
                               f"U{{1e-6,1e-9}}, CFIE D-ikS, seed 0",
                   "patches": bs.n_patches, "points": bs.n_points,
                   "value": bs.n_points / (bms / 1e3), "unit": UNIT, "ms_per_step": bms,
                   "launches_per_step": int(b_launches), "status": st_b,
                   "one_by_one": {"value": bs.n_points / (one_ms / 1e3), "ms": one_ms,
                                  "launches": int(one_launches)},
                   "mixed": {"value": bs.n_points / (bm_ms / 1e3), "unit": UNIT,
                             "ms_per_step": bm_ms, "status": st_bm,
                             "pair_form": FORM_NAMES[bm_forms]}}
        del bds, bx_d, btn_d

    # the paper's Table 1 on its twisted torus (2400 patches, S, k = 1): oversampling
    # alpha = N_over / N, stored corrections per point m = nnz / N and S_init = N / T_init
    # for p = d + 1 in {2, 3, 4, 6, 8} and eps in {5e-3, 5e-4, 5e-7, 5e-10}
    table1 = None
    if not args.no_variants and not args.no_table1:
        table1 = []
        for d in (1, 2, 3, 5, 7):
            ts = W.stellarator(20, 60, d)
            tx, ttn = W.onsurface_targets(ts)
            tds = lcq.DeviceSurface(ts.deg, ts.node_off, torch.from_numpy(ts.xyz).to(dev))
            tx_d1 = torch.from_numpy(tx).to(dev)
            ttn_d1 = torch.from_numpy(ttn).to(dev)
            for eps in (5e-3, 5e-4, 5e-7, 5e-10):
                tp = lcq.params(eps, test_dirs=W.test_directions(7))
                ms = []
                for it in range(TUNING_GENERATIONS + 2):   # tuner candidates, warm-up, timed
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    near = lcq.build_near_lists(ctx, tds, tx_d1, ttn_d1, tp)
                    corr = lcq.gen_corrections(ctx, tds, near, "S", 1.0, tp)
                    e1.record(stream)
                    st_t = ctx.sync()
                    ms.append(e0.elapsed_time(e1))
                    t_stages = ctx.stage_times()[0]
                    t_group = int(ctx.counters()[5])
                    nnz, n_over = corr.info()
                    corr.close()
                    near.close()
                table1.append({"p": d + 1, "eps": eps, "points": ts.n_points,
                               "alpha": n_over / ts.n_points, "m": nnz / ts.n_points,
                               "S_init": ts.n_points / (ms[-1] / 1e3), "status": st_t,
                               "group_size": t_group,
                               "stages_ms": [round(float(x), 3) for x in t_stages]})
            del tds, tx_d1, ttn_d1

    # the paper's Table 2 (performance against the patches' aspect ratio); a failure is
    # recorded in the line rather than ending the run
    table2 = None
    if not args.no_variants and not args.no_table2:
        try:
            table2 = table2_sweep(ctx, lcq, W, dev, stream, flush)
        except Exception as exc:  # noqa: BLE001
            table2 = {"error": repr(exc)}

    # the 40,000-patch torus (k = 20, eps = 1e-9), FP64 and mixed, one timed step each; the
    # two CSRs are compared on the device; then the corrected potential at a 100,000-point
    # subset of the nodes (its own near lists and corrections, and the direct far sum over
    # every oversampled source), the apply timed alone
    large = None
    if not args.no_large and not args.no_variants:
        lw = W.torus_cfie_k20(100)
        ls = lw.surface
        lds = lcq.DeviceSurface(ls.deg, ls.node_off, torch.from_numpy(ls.xyz).to(dev))
        lx = torch.from_numpy(lw.tgt_xyz).to(dev)
        ltn = torch.from_numpy(lw.tgt_node).to(dev)
        lp = lcq.params(lw.eps, test_dirs=W.test_directions(7))
        large, vals = {"workload": lw.name, "patches": ls.n_patches, "points": ls.n_points}, {}
        for prec in ("fp64", "mixed"):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            near = lcq.build_near_lists(ctx, lds, lx, ltn, lp)
            corr = lcq.gen_corrections(ctx, lds, near, lw.kernel, lw.k, lp, lw.alpha, lw.beta,
                                       precision=prec)
            e1.record(stream)
            st_l = ctx.sync()
            ms = e0.elapsed_time(e1)
            nnz = near.nnz
            dv = torch.empty(nnz, dtype=torch.complex128, device=dev)
            corr.export(ls.n_points, out=(None, None, dv))
            vals[prec] = dv
            forms = int(ctx.counters()[7])
            large[prec] = {"value": ls.n_points / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
                           "status": st_l, "nnz": nnz,
                           "adaptive_ms": ctx.stage_times()[0][3],
                           "pair_form": FORM_NAMES[forms], "fp32_used": forms != 0}
            corr.close()
            near.close()
        large["mixed"]["csr_rel_l2_vs_fp64"] = float(
            torch.linalg.vector_norm(vals["mixed"] - vals["fp64"]) /
            torch.linalg.vector_norm(vals["fp64"]))

        del vals
        sub = np.arange(0, ls.n_points, ls.n_points // 100000)[:100000]
        sx = torch.from_numpy(np.ascontiguousarray(lw.tgt_xyz[:, sub])).to(dev)
        stn = torch.from_numpy(np.ascontiguousarray(lw.tgt_node[sub])).to(dev)
        near = lcq.build_near_lists(ctx, lds, sx, stn, lp)
        corr = lcq.gen_corrections(ctx, lds, near, lw.kernel, lw.k, lp, lw.alpha, lw.beta)
        sig = torch.from_numpy(W.density(ls.n_points, 0)).to(dev)
        ctx.sync()   # one timed apply: a minute-long launch needs no warm-up
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        u = lcq.apply_corrected_CFIE(ctx, lds, near, corr, sig, len(sub))
        e1.record(stream)
        st_a = ctx.sync()
        nnz_s, n_over = corr.info()
        large["apply_100k"] = {"targets": len(sub), "sources_oversampled": n_over,
                               "ms": e0.elapsed_time(e1), "status": st_a,
                               "finite": bool(torch.isfinite(u).all())}
        corr.close()
        near.close()
        del lds, lx, ltn, sx, stn, sig, u

    # end to end through the C ABI with host buffers: H2D of inputs, D2H of the CSR
    e2e = None
    if not args.no_e2e:
        xyz_h = torch.from_numpy(surf.xyz).pin_memory()
        tx_h = torch.from_numpy(np.ascontiguousarray(wl.tgt_xyz)).pin_memory()
        tn_h = torch.from_numpy(wl.tgt_node).pin_memory()
        near, corr = step()
        nnz = near.nnz
        corr.close()
        near.close()
        rp_h = torch.empty(NT + 1, dtype=torch.int64).pin_memory()
        col_h = torch.empty(nnz, dtype=torch.int32).pin_memory()
        val_h = torch.empty(nnz, dtype=torch.complex128).pin_memory()
        out = (rp_h.numpy(), col_h.numpy(), val_h.numpy())
        xyz_e = torch.empty_like(xyz_d)
        tx_e = torch.empty_like(tx_d)
        tn_e = torch.empty_like(tn_d)
        ds_e = lcq.DeviceSurface(surf.deg, surf.node_off, xyz_e)
        e2e_t = []
        for it in range(args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            with torch.cuda.stream(stream):
                xyz_e.copy_(xyz_h, non_blocking=True)
                tx_e.copy_(tx_h, non_blocking=True)
                tn_e.copy_(tn_h, non_blocking=True)
            near = lcq.build_near_lists(ctx, ds_e, tx_e, tn_e, prm)
            corr = lcq.gen_corrections(ctx, ds_e, near, wl.kernel, wl.k, prm, wl.alpha, wl.beta)
            corr.export(NT, out=out)
            t1 = time.perf_counter()
            corr.close()
            near.close()
            if it >= args.warmup:
                e2e_t.append(t1 - t0)
        tot = max_over_ranks(sum(e2e_t), dev)
        e2e = {"value": job_throughput(N, len(e2e_t), world, tot * 1e3), "unit": UNIT,
               "h2d_bytes_per_step": int(xyz_h.numel() * 8 + tx_h.numel() * 8 + tn_h.numel() * 8),
               "d2h_bytes_per_step": int((NT + 1) * 8 + nnz * 4 + nnz * 16)}

    if rank != 0:
        return
    fpe = flops_per_eval(n)
    flops = nodes * fpe
    a_ms = statistics.mean(adapt_ms)
    achieved = flops / (a_ms / 1e3) / 1e12
    peak = peaks["fp64_fma_tflops"]
    roofline = {"bound": "alu",
                "kernel": ("k_adaptive<6>: " + {"fp64": "FP64", "fp32": "FP32",
                                                 "two-float": "two-float"}.get(
                               FORM_NAMES[main_forms], "mixed") +
                           " kernel values, FP64 geometry; contraction on the f16 tensor "
                           "cores by an exact slice split"),
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic_for("k_adaptive"),
                "peak_source": "measured in this run: FP64 FMA chains on every SM "
                               "(lcq_pipe_peaks), CUDA events",
                "flops_per_eval": fpe,
                "flops_per_eval_terms": "20 arithmetic + 3 special functions (sqrt, reciprocal, "
                                        "sincos) + 4n contraction, n = 28",
                "flops_per_launch": flops, "node_evals_per_launch": nodes,
                "tests_per_launch": tests, "union_tree_nodes_per_launch": tree_nodes,
                "work_items_per_launch": items, "targets_per_item_max": group_size,
                "avg_launch_ms": a_ms}
    cpu = None
    if not args.no_cpu_baseline:
        workers = max(1, min(16, os.cpu_count() or 1))
        pool = make_pool(workers)
        v, done, worst = oracle_sample(args.s, P, workers, 1, 0, pool, args.eps, args.leaf_order)
        pool.close()
        # one core, beside the paper's single-core figures: median of 3 samples of 2 patches
        pool1 = make_pool(1)
        one = [oracle_sample(args.s, P, 1, 2, 101 * r, pool1, args.eps, args.leaf_order)[0]
               for r in range(3)]
        pool1.close()
        cpu = {"value": v, "unit": UNIT, "cores": workers, "kind": "oracle",
               "sample": f"{done} of {P} patches (1 per worker, spread over the surface); "
                         f"sampled points / slowest worker's compute time ({worst:.1f} s)",
               "single_core": {"value": statistics.median(one), "unit": UNIT, "cores": 1,
                               "sample": "median of 3 samples of 2 patches each, one process",
                               "samples": one}}
    st_mean = [statistics.mean(s[i] for s in stages) for i in range(6)]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else MIXED_DTYPE[FORM_NAMES[main_forms]],
        "data": "synthetic",
        "config": {"workload": workload_name(P, N, args.eps, args.precision), "patches": P,
                   "order": 6, "precision": args.precision,
                   "points": N, "eps": args.eps, "leaf_order": args.leaf_order or "q_j",
                   "l2": "256 MiB buffer written between steps (outside the timed events)",
                   "tuning": f"{TUNING_GENERATIONS} untimed generations before the warm-up "
                             f"time the group-size tuner's candidates"},
        "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
        "pipe_peaks": peaks,
        "clocks": clk, "status": max(statuses) if statuses else None,
        "stages_ms": dict(zip(["near_lists", "far_order", "smooth_annulus", "adaptive", "self",
                               "v2c"], st_mean)),
        "variants": variants,
        "sphere20": small,
        "batched": batched,
        "table1": table1,
        "table2": table2,
        "large": large,
        "wall_s_timed_region": t_wall,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    if args.impl == "reference":
        run_reference(args, rank)
    else:
        run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
