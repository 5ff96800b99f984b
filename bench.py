#!/usr/bin/env python3
"""Benchmark of SIVF spherical k-means on GB300.

Workload (default): the medium single-GPU corpus, N = 300,000 documents,
D = 100,000 terms, Zipf s = 1.05, lognormal(5.0, 0.7) lengths clipped to
[10, 3000] (~190 nnz/doc, 57M nnz), k = 1000, FP32 postings, ICP on.

A step is one complete clustering run from the seeded initial centroids:
seeding + up to 50 Lloyd iterations (assignment, Algorithm 4, and update,
Algorithm 5), every step identical. `value` = objects assigned per second
(N * iterations / step time), inputs resident in HBM; `e2e` = the same metric
through the C ABI with the corpus in pinned host memory and the labels copied
back, every step.

--impl reference times the FP64 CPU oracle (the plain restatement of the
method) on the host cores instead: each step is one Lloyd iteration of the
same workload.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from synth import CONFIGS, generate, init_ids  # noqa: E402

# bytes per posting read by the scan: 16-bit id + value (k <= 65536), else 32-bit id + value
B_POST16 = {"fp32": 6, "bf16": 4, "fp16": 4}
B_POST32 = {"fp32": 8, "bf16": 6, "fp16": 6}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2", choices=sorted(CONFIGS) + ["c4"])
    ap.add_argument("--precision", default=None, choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--icp", type=int, default=1, choices=[0, 1, 2, 3],
                    help="1: SIVF (Algorithm 4); 0: unfiltered IVF (Algorithm 2); 2: IVF-CBICP (Algorithm 3); "
                         "3: SIVF with the relaxed filter")
    ap.add_argument("--max-iter", type=int, default=None)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--graph", type=int, default=1, help="1: iterations after the second run in one CUDA graph")
    ap.add_argument("--autotune", type=int, default=1, help="1: pick the assignment kernel configuration by timing")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-iters", type=int, default=8)
    return ap.parse_args()


def recorded_traffic(w):
    """DRAM bytes of one assignment launch from a committed ncu capture, if the
    kernel source is unchanged since the capture (else None)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", f"assign_kernel_{w.name}_{w.precision}.json")
    src = os.path.join(ROOT, "paper_2103_16141_gb300", "csrc", "assign.cu")
    try:
        rec = json.load(open(path))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except Exception:
        return None, None
    if rec.get("source_sha256") != sha:
        return None, None
    return float(rec["dram_bytes_per_launch"]), rec


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier_and_sync(world):
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    if torch.cuda.is_available():
        torch.cuda.synchronize()


def _reduce(x, world, op):
    """All-reduce of one host scalar over the ranks (device tensor under NCCL,
    host tensor under gloo)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, world):
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.MAX) if world > 1 else x


def sum_over_ranks(x, world):
    import torch.distributed as dist
    return _reduce(x, world, dist.ReduceOp.SUM) if world > 1 else x


def replica_throughput(units_local, ms_local, world):
    """Whole-job throughput of independent replicas: the units every rank
    processed over the slowest rank's time (ms). Returns (units/s, max ms)."""
    ms = max_over_ranks(ms_local, world)
    return sum_over_ranks(float(units_local), world) / (ms / 1e3), ms


def cpu_baseline(w, c, ini, iters, icp=1):
    """The FP64 oracle (OpenMP, all host cores) on a bounded sample of the same
    workload: the first `iters` Lloyd iterations (assign + update), in the
    same assignment algorithm."""
    from oracle import Oracle
    o = Oracle(c, w.k, ini, icp=icp)
    t0 = time.perf_counter()
    done = 0
    for _ in range(iters):
        a = o.assign()
        done += 1
        if a.r > 1 and a.changed == 0:
            break
        o.update()
    dt = time.perf_counter() - t0
    cores = Oracle.threads()
    out = {"value": w.N * done / dt, "unit": "objects/s", "cores": cores, "kind": "oracle",
           "sample": f"first {done} Lloyd iterations (assign+update) of the same corpus, FP64 oracle, "
                     f"{dt:.1f} s", "sec_per_iter": dt / done}
    # one thread, first iteration only (bounded): the per-core figure
    o1 = Oracle(c, w.k, ini, icp=icp, threads=1)
    try:
        t1 = time.perf_counter()
        o1.assign()
        o1.update()
        d1 = time.perf_counter() - t1
    finally:
        Oracle(c, w.k, ini, icp=icp, threads=cores)  # restore the thread count
    t0 = time.perf_counter()
    o2 = Oracle(c, w.k, ini, icp=icp)
    o2.assign()
    o2.update()
    d2 = time.perf_counter() - t0
    out["single_thread"] = {"value": w.N / d1, "unit": "objects/s", "sample": "iteration 1, one thread",
                            "same_sample_all_cores": w.N / d2}
    return out


L2_BYTES = 129 * 2**20  # GB300 L2
METRIC = "objects/s (Lloyd iterations of SIVF spherical k-means); sec per Lloyd iteration"
ICP_NAMES = ["ivf", "sivf", "ivf-cbicp", "sivf-relaxed"]


def workload_name(w, nnz: int) -> str:
    """The workload as both arms name it in config.workload."""
    return (f"{w.name}: N={w.N} D={w.D} nnz={nnz} k={w.k} zipf={w.zipf_s} "
            f"len=lognormal({w.mu:.3f},{w.sigma}) clip[{w.lo},{w.hi}] seed={w.seed}")


def run_reference(args, w):
    """Reference arm: the FP64 CPU oracle, each step one Lloyd iteration."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    from oracle import Oracle
    c = generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, w.seed)
    ini = init_ids(w.N, w.k, w.init_seed)
    o = Oracle(c, w.k, ini, icp=args.icp)

    def step():
        a = o.assign()
        if a.r > 1 and a.changed == 0:
            o.set_labels(o.labels())
        o.update()

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = w.N * args.steps / dt
    line = {"metric": METRIC, "value": value, "unit": "objects/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_name(w, c.nnz), "icp": ICP_NAMES[args.icp], "max_iter": w.max_iter,
                       "iters_per_step": 1},
            "cpu_baseline": {"value": value, "unit": "objects/s", "cores": Oracle.threads(), "kind": "oracle",
                             "sample": f"iterations {args.warmup + 1}..{args.warmup + args.steps} of the corpus"},
            "e2e": {"value": value, "unit": "objects/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_batched(args):
    """Batched workload: 64 independent corpora (seeds 0..63; N log-uniform in
    [5K, 200K], D in [20K, 100K], mean nnz/doc in [30, 250], k in [16, 2000]),
    FP16 postings, one context; a step is one sivf_batch_run to convergence
    (cap 50) from the seeded centroids."""
    import torch
    from paper_2103_16141_gb300 import SIVFBatch, sivf as S
    from synth import batched_instances

    world, rank, local = dist_setup(args.gpus)
    S.load()
    prec = args.precision or "fp16"
    ws = batched_instances(64, max_iter=args.max_iter or 50)
    cs = [generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, w.seed) for w in ws]
    inis = [init_ids(w.N, w.k, w.init_seed) for w in ws]
    b = SIVFBatch(cs, [w.k for w in ws], inis, precision=prec, icp=args.icp, threads=args.threads,
                  ctas_per_sm=args.ctas_per_sm, use_graph=bool(args.graph), autotune=bool(args.autotune))
    gini = np.ascontiguousarray(np.concatenate([ini + off for ini, off in
                                                zip(inis, np.cumsum([0] + [w.N for w in ws[:-1]]))]), dtype=np.int32)
    max_iter = ws[0].max_iter
    stream = torch.cuda.current_stream()

    def one_run():
        S.sivf_reseed(b.ctx, gini.ctypes.data)  # gini stays referenced during the call
        its, _ = b.run(max_iter)
        return its, b.stats()

    for _ in range(args.warmup):
        one_run()
    sampler = ClockSampler(local)
    sampler.start()
    barrier_and_sync(world)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    obj_iters = 0
    launches = 0
    for _ in range(args.steps):
        its, st = one_run()
        obj_iters += int(sum(w.N * int(i) for w, i in zip(ws, its)))
        launches += st["launches"]
    ev1.record(stream)
    barrier_and_sync(world)
    clocks = sampler.stop()
    value, ms = replica_throughput(obj_iters, ev0.elapsed_time(ev1), world)
    if rank == 0:
        nnz = sum(c.nnz for c in cs)
        line = {"metric": "objects/s (Lloyd iterations of SIVF spherical k-means, 64 batched instances)",
                "value": value, "unit": "objects/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": f"{prec}-postings/f32-products/fixed-point-sum", "data": "synthetic",
                "config": {"workload": f"c4: 64 instances, N={sum(w.N for w in ws)} total, nnz={nnz}, "
                                       f"k={sum(w.k for w in ws)} total, max k={max(w.k for w in ws)}",
                           "iterations_per_instance": [int(i) for i in its], "max_iter": max_iter},
                "gpu_launches": int(launches), "clocks": clocks}
        print(json.dumps(line), flush=True)
    b.close()


def main():
    args = parse()
    if args.config == "c4":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no CPU reference arm"}))
            return
        run_batched(args)
        return
    w = CONFIGS[args.config]
    if args.precision:
        w = w.scaled(precision=args.precision)
    if args.max_iter:
        w = w.scaled(max_iter=args.max_iter)
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    from paper_2103_16141_gb300 import SIVF, sivf as S

    world, rank, local = dist_setup(args.gpus)
    S.load()
    # each rank is an independent replica of the workload (the path needs no exchange)
    c = generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, w.seed)
    ini = init_ids(w.N, w.k, w.init_seed)
    dev = torch.device("cuda", torch.cuda.current_device())
    g = SIVF(c.row_ptr, c.idx, c.val, c.D, w.k, ini, precision=w.precision, icp=args.icp,
             threads=args.threads, ctas_per_sm=args.ctas_per_sm, use_graph=bool(args.graph),
             autotune=bool(args.autotune))
    stream = torch.cuda.current_stream()

    def one_run_stepped():
        """Host-stepped run: per-iteration counters and per-launch device times."""
        g.reseed(ini)
        iters = 0
        per = []
        for _ in range(w.max_iter):
            n = g.assign()
            iters += 1
            st = g.stats()
            per.append(st)
            if st["iter"] > 1 and n == 0:
                break
            g.update()
            per[-1] = {**st, "ms_update": g.stats()["ms_update"], "centroid_nnz": g.stats()["centroid_nnz"]}
        per[-1]["launches_run"] = g.stats()["launches"]  # reseed resets the count
        return iters, per

    def one_run_graph():
        g.reseed(ini)
        iters, _ = g.run(w.max_iter)
        return iters, [{"launches_run": g.stats()["launches"]}]

    one_run = one_run_graph if args.graph else one_run_stepped

    for _ in range(args.warmup):
        one_run()

    sampler = ClockSampler(local)
    sampler.start()
    barrier_and_sync(world)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    tot_iters, all_per = 0, []
    for _ in range(args.steps):
        it, per = one_run()
        tot_iters += it
        all_per.extend(per)
    ev1.record(stream)
    barrier_and_sync(world)
    clocks = sampler.stop()
    launches = sum(p["launches_run"] for p in all_per if "launches_run" in p)
    value, ms = replica_throughput(w.N * tot_iters, ev0.elapsed_time(ev1), world)

    # roofline of the dominant kernel (the assignment scan), from the library's
    # per-launch event timings: over the timed region when steps are launched
    # from the host, else over one host-stepped run of the same workload
    kernel_times_from = "timed region"
    if args.graph:
        _, all_per = one_run_stepped()
        kernel_times_from = "one host-stepped run of the same workload (graph replay hides per-launch times)"
    hbm_peak, peak_src = load_peaks()
    b_post = (B_POST16 if w.k <= 65536 else B_POST32)[w.precision]
    fixed = c.nnz * 8 + (w.N + 1) * 8 + w.N * 16 + w.k
    alg_bytes = sum(fixed + p["postings"] * b_post for p in all_per)
    # compulsory bytes: every posting of the scanned file read once (the file
    # of iteration r is built by update r-1; the first one holds the seed rows)
    seed_nnz = int(sum(c.row_ptr[i + 1] - c.row_ptr[i] for i in ini))
    if_nnz = [seed_nnz] + [p.get("centroid_nnz", 0) for p in all_per[:-1]]
    min_bytes = sum(fixed + n * b_post for n in if_nnz)
    ms_assign = sum(p["ms_assign"] for p in all_per)
    ms_update = sum(p.get("ms_update", 0.0) for p in all_per)
    stepped_iters = len(all_per)
    achieved = alg_bytes / (ms_assign / 1e3) / 1e9 if ms_assign > 0 else 0.0
    postings = sum(p["postings"] for p in all_per)
    simcalc = sum(p["simcalc"] for p in all_per)
    iters_per_step = tot_iters / args.steps
    traffic, trec = recorded_traffic(w)

    # end to end: host corpus in pinned memory -> device, init, run, labels back
    e2e = None
    if not args.no_e2e:
        # the C ABI copies the pinned host CSR itself (inputs_on_host)
        rp = torch.from_numpy(c.row_ptr).pin_memory()
        ix = torch.from_numpy(c.idx).pin_memory()
        vl = torch.from_numpy(c.val).pin_memory()
        lab_host = torch.empty(w.N, dtype=torch.int32).pin_memory()
        h2d = rp.numel() * 8 + ix.numel() * 4 + vl.numel() * 4
        d2h = w.N * 4
        barrier_and_sync(world)
        t0 = time.perf_counter()
        e_iters = 0
        E = max(1, min(args.steps, 3))
        for _ in range(E):
            ge = SIVF(rp, ix, vl, c.D, w.k, ini, precision=w.precision, icp=args.icp,
                      threads=args.threads, ctas_per_sm=args.ctas_per_sm, use_graph=bool(args.graph),
                      autotune=bool(args.autotune), inputs_on_host=True)
            it, _ = ge.run(w.max_iter)
            e_iters += it
            S.sivf_get_labels(ge.ctx, lab_host.data_ptr(), False)
            ge.close()
        barrier_and_sync(world)
        dt = max_over_ranks(time.perf_counter() - t0, world)
        e2e = {"value": sum_over_ranks(float(w.N * e_iters), world) / dt, "unit": "objects/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": E}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, c, ini, args.cpu_sample_iters, args.icp)

    if rank == 0:
        csr_bytes = c.nnz * 8 + (w.N + 1) * 8
        line = {
            "metric": METRIC,
            "value": value, "unit": "objects/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if w.precision == "fp32" else f"{w.precision}-postings/f32-products/fixed-point-sum",
            "data": "synthetic",
            "config": {"workload": workload_name(w, c.nnz),
                       "precision": w.precision, "icp": ICP_NAMES[args.icp], "max_iter": w.max_iter,
                       "iters_per_step": iters_per_step, "sec_per_iter": ms / 1e3 / tot_iters,
                       "l2": (f"inputs larger than L2: every assignment streams the object CSR "
                              f"({csr_bytes / 1e9:.2f} GB); the inverted file is reused from L2 within a launch"
                              if csr_bytes > L2_BYTES else
                              f"inputs fit in L2 ({csr_bytes / 1e6:.1f} MB CSR), no flush: a small-case timing, "
                              f"not the workload of record"),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "cuda_graph": bool(args.graph), "autotune": bool(args.autotune),
                       "assign_threads": g.stats()["assign_threads"],
                       "score_buffer": "global" if g.stats()["assign_global"] else "shared"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                         "frac": achieved / hbm_peak, "traffic": traffic,
                         "traffic_launch": trec.get("launch") if trec else None,
                         "peak_source": peak_src, "kernel": "assign_kernel",
                         "bytes_model": f"nnz*8 + (N+1)*8 + postings*b_post + N*16 + k, b_post = {b_post} B "
                                        f"(no cache credit)",
                         "note": "posting bytes are served by L2, not HBM (traffic = ncu DRAM bytes of one "
                                 "launch); frac > 1 means on-chip reuse, see profiles/",
                         "compulsory_frac": min_bytes / (ms_assign / 1e3) / 1e9 / hbm_peak if ms_assign > 0 else None,
                         "ncu_dram_gbs": (traffic / trec["ncu_duration_s"] / 1e9) if trec else None,
                         "postings_per_s": postings / (ms_assign / 1e3) if ms_assign > 0 else None,
                         "simcalc_ratio": simcalc / (float(w.N) * w.k * stepped_iters),
                         "ms_assign_per_iter": ms_assign / stepped_iters, "ms_update_per_iter": ms_update / stepped_iters,
                         "kernel_times_from": kernel_times_from},
            "per_iteration": {"postings": [int(p["postings"]) for p in all_per[:60]],
                              "filtered": [int(p["filtered"]) for p in all_per[:60]],
                              "rescored": [int(p["rescored"]) for p in all_per[:60]],
                              "ms_assign": [round(p["ms_assign"], 3) for p in all_per[:60]],
                              "ms_update": [round(p.get("ms_update", 0.0), 3) for p in all_per[:60]]},
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        if e2e:
            line["e2e"] = e2e
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    g.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
