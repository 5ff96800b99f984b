#!/usr/bin/env python3
"""Benchmark of SIVF spherical k-means on GB300.

Workload (default): the largest single-GPU corpus, N = 8,000,000 documents,
D = 140,000 terms, Zipf s = 1.1, lognormal lengths of mean 60 (sigma 0.8,
clipped to [5, 3000]; 480M nnz, 3.84 GB CSR), k = 20,000, BF16 postings with
the exact re-score, ICP on.

A step is one Lloyd iteration (assignment, Algorithm 4, then update,
Algorithm 5) with the state carried from step to step: the W warm-up steps are
iterations 1..W from the seeded centroids and the K timed steps are iterations
W+1..W+K (the iteration cap of the workload does not stop the window). `value` =
objects assigned per second (N * K / timed seconds), inputs resident in HBM,
CUDA events on the library's stream. Beside it:
  - vs_fp32: the same window with FP32 postings, in the same process (both
    paths re-score every object whose top-2 margin lies inside their error
    bound exactly, so their labels are the same at every iteration, checked);
  - roofline of the assignment kernel for both paths, against the measured
    L2-read or HBM peak, whichever serves most of its algorithmic bytes;
  - e2e: the same window through the C ABI with the CSR copied from pinned
    host memory and the labels read back, every step;
  - cpu_baseline: the FP64 oracle on the host cores, on a bounded sample.

--impl reference times the FP64 CPU oracle (the plain restatement of the
method) on the same workload and window instead.
"""
from __future__ import annotations

import argparse
import hashlib
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

# bytes per posting read by the sparse scan: 16-bit id + value (k <= 65536), else 32-bit id + value
B_POST16 = {"fp32": 6, "bf16": 4, "fp16": 4}
B_POST32 = {"fp32": 8, "bf16": 6, "fp16": 6}
# bytes per entry of a dense head-term row
B_DENSE = {"fp32": 4, "bf16": 2, "fp16": 2}
L2_BYTES = 129 * 2**20  # GB300 L2
METRIC = "objects/s (Lloyd iterations of SIVF spherical k-means); sec per Lloyd iteration"
ICP_NAMES = ["ivf", "sivf", "ivf-cbicp", "sivf-relaxed"]
REF_SAMPLE = 2048  # objects scored per sampled oracle step


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c5", choices=sorted(CONFIGS) + ["c4"])
    ap.add_argument("--precision", default=None, choices=["fp32", "bf16", "fp16"])
    ap.add_argument("--icp", type=int, default=1, choices=[0, 1, 2, 3],
                    help="1: SIVF (Algorithm 4); 0: unfiltered IVF (Algorithm 2); 2: IVF-CBICP (Algorithm 3); "
                         "3: SIVF with the relaxed filter")
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    ap.add_argument("--autotune", type=int, default=1, help="1: pick the assignment kernel configuration by timing")
    ap.add_argument("--graph", type=int, default=1, help="c4 only: iterations after the second in one CUDA graph")
    ap.add_argument("--max-iter", type=int, default=None, help="c4 only: iteration cap of each instance")
    ap.add_argument("--dense-max-mb", type=float, default=0.0,
                    help="device memory for dense head-term rows (0 = automatic, < 0 = none)")
    ap.add_argument("--dense-min-fraction", type=float, default=0.0,
                    help="list length / k from which a term gets a dense row (0 = automatic)")
    ap.add_argument("--dense-all", action="store_true",
                    help="every term from a dense row: the dense-mean variant (Lloyd-ICP with dense means)")
    ap.add_argument("--light-max-moving", type=int, default=0,
                    help="warp-per-object path up to this many moving clusters (0 = automatic, < 0 = off)")
    ap.add_argument("--update-mode", default="auto", choices=["auto", "dense", "sort"],
                    help="cluster sums of the update step (sort: no k x D accumulator, for small captures)")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32 comparison path")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=0, help="timed e2e steps (0 = --steps: the same window)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def recorded_traffic(w, prec):
    """DRAM bytes of one assignment launch from a committed ncu summary, if
    the kernel source is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", f"assign_kernel_{w.name}_{prec}.json")
    src = os.path.join(ROOT, "paper_2103_16141_gb300", "csrc", "assign.cu")
    try:
        rec = json.load(open(path))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except Exception:
        return None
    if rec.get("source_sha256") != sha:
        return None
    return rec


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


def workload_name(w, nnz: int) -> str:
    """The workload as both arms name it in config.workload."""
    return (f"{w.name}: N={w.N} D={w.D} nnz={nnz} k={w.k} zipf={w.zipf_s} "
            f"len=lognormal({w.mu:.3f},{w.sigma}) clip[{w.lo},{w.hi}] seed={w.seed}")


def shared_config(w, nnz, args):
    """The `config` both arms print (identical dicts for the same workload)."""
    csr_bytes = nnz * 8 + (w.N + 1) * 8
    return {"workload": workload_name(w, nnz),
            "window": f"iterations {args.warmup + 1}-{args.warmup + args.steps} of one run from the seeded "
                      f"centroids (warm-up iterations 1-{args.warmup}); one step = one Lloyd iteration",
            "l2": (f"inputs larger than L2: every assignment streams the object CSR ({csr_bytes / 1e9:.2f} GB)"
                   if csr_bytes > L2_BYTES else
                   f"inputs fit in L2 ({csr_bytes / 1e6:.1f} MB CSR), no flush: a small-case timing")}


# ---------------------------------------------------------------- oracle arm

def sampled_reference_state(c, w, ini):
    """FP64 oracle holding centroids of realistic density for sampled scoring:
    the means of a seeded balanced labelling (every cluster N/k members)."""
    from oracle import Oracle
    o = Oracle(c, w.k, ini, icp=False)
    rng = np.random.default_rng(w.seed + 77)
    lab = (rng.permutation(w.N) % w.k).astype(np.int32)
    o.set_labels(lab)
    o.update()
    return o


def sampled_oracle_step(o, w, step):
    """One sampled oracle iteration: REF_SAMPLE seeded objects scored against
    all k centroids (Algorithm 2 scoring, FP64), then one full update step.
    Returns (measured seconds, estimated seconds of a whole iteration)."""
    rng = np.random.default_rng(1000 + step)
    ids = np.sort(rng.choice(w.N, size=min(REF_SAMPLE, w.N), replace=False)).astype(np.int64)
    t0 = time.perf_counter()
    o.score_objects(ids)
    t1 = time.perf_counter()
    o.update()
    t2 = time.perf_counter()
    return t2 - t0, (t1 - t0) * w.N / len(ids) + (t2 - t1)


def full_oracle_iterations(c, w, ini, icp):
    """Generator of whole oracle Lloyd iterations (assign + update), seconds each."""
    from oracle import Oracle
    o = Oracle(c, w.k, ini, icp=icp)
    while True:
        t0 = time.perf_counter()
        a = o.assign()
        if a.r > 1 and a.changed == 0:  # converged: restart from the seeds
            o = Oracle(c, w.k, ini, icp=icp)
            a = o.assign()
        o.update()
        yield time.perf_counter() - t0


def oracle_is_sampled(w) -> bool:
    return float(w.N) * w.k > 1e9  # whole iterations only for the small and medium corpora


def run_reference(args, w):
    """Reference arm: the FP64 CPU oracle on the same workload and window."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    from oracle import Oracle
    c = generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, w.seed)
    ini = init_ids(w.N, w.k, w.init_seed)
    if oracle_is_sampled(w):
        o = sampled_reference_state(c, w, ini)
        for s in range(args.warmup):
            sampled_oracle_step(o, w, s)
        meas, est = 0.0, 0.0
        for s in range(args.steps):
            m, e = sampled_oracle_step(o, w, args.warmup + s)
            meas += m
            est += e
        value = w.N * args.steps / est
        ms_step = meas / args.steps * 1e3
        sample = (f"per step: {REF_SAMPLE} seeded objects scored in FP64 against all k centroids (unfiltered, "
                  f"Algorithm 2 scoring; time scaled by N/{REF_SAMPLE}) plus one whole update step; the "
                  f"centroids are the means of a seeded balanced labelling (N/k members each), since the oracle "
                  f"cannot run whole iterations of this corpus; ms_per_step is the measured sample time, value "
                  f"the estimated whole iterations: {est / args.steps:.1f} s each")
    else:
        it = full_oracle_iterations(c, w, ini, args.icp)
        for _ in range(args.warmup):
            next(it)
        t = sum(next(it) for _ in range(args.steps))
        value = w.N * args.steps / t
        ms_step = t / args.steps * 1e3
        sample = f"iterations {args.warmup + 1}..{args.warmup + args.steps} of the corpus, whole Lloyd iterations"
    line = {"metric": METRIC, "value": value, "unit": "objects/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference", "config": shared_config(w, c.nnz, args),
            "cpu_baseline": {"value": value, "unit": "objects/s", "cores": Oracle.threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "objects/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(w, c, ini, icp):
    """The FP64 oracle (OpenMP, all host cores) on a bounded sample of the same
    workload (about 10-30 s of CPU work)."""
    from oracle import Oracle
    cores = Oracle.threads()
    if oracle_is_sampled(w):
        o = sampled_reference_state(c, w, ini)
        meas = est = 0.0
        steps = 2
        for s in range(steps):
            m, e = sampled_oracle_step(o, w, s)
            meas += m
            est += e
        return {"value": w.N * steps / est, "unit": "objects/s", "cores": cores, "kind": "oracle",
                "sample": f"{steps} sampled iterations: {REF_SAMPLE} seeded objects scored in FP64 against all k "
                          f"centroids (scaled by N/{REF_SAMPLE}) plus one whole update step each, {meas:.1f} s "
                          f"measured", "sec_per_iter": est / steps}
    it = full_oracle_iterations(c, w, ini, icp)
    t, done = 0.0, 0
    while done < 8 and t < 20.0:
        t += next(it)
        done += 1
    return {"value": w.N * done / t, "unit": "objects/s", "cores": cores, "kind": "oracle",
            "sample": f"first {done} Lloyd iterations (assign+update) of the same corpus, FP64 oracle, {t:.1f} s",
            "sec_per_iter": t / done}


# ---------------------------------------------------------------- CUDA arm

def measure_peaks(dev, stream):
    """Streaming-read bandwidth measured here with CUDA events: a 64 MB buffer
    (L2-resident) and a 4 GB one (HBM)."""
    import torch
    from paper_2103_16141_gb300 import sivf as S
    out = {}
    for name, nbytes, passes in (("l2", 64 << 20, 400), ("hbm", 4 << 30, 5)):
        buf = torch.zeros(nbytes // 4, dtype=torch.int32, device=dev)
        best = 0.0
        for _ in range(3):
            gbs, _ = S.sivf_measure_read_bandwidth(buf.data_ptr(), nbytes, passes, stream.cuda_stream)
            best = max(best, gbs)
        out[name] = best
        del buf
    torch.cuda.empty_cache()
    return out


class Path:
    """One clustering run stepped one Lloyd iteration at a time."""

    def __init__(self, c, csr, w, ini, precision, args):
        from paper_2103_16141_gb300 import SIVF
        self.w, self.ini = w, ini
        rp, ix, vl = csr
        self.g = SIVF(rp, ix, vl, c.D, w.k, ini, precision=precision, icp=args.icp, threads=args.threads,
                      ctas_per_sm=args.ctas_per_sm, autotune=bool(args.autotune),
                      dense_max_bytes=int(args.dense_max_mb * 2**20) if args.dense_max_mb >= 0 else -1,
                      dense_min_fraction=args.dense_min_fraction, update_mode=args.update_mode,
                      dense_all=args.dense_all, light_max_moving=args.light_max_moving)
        self.converged = False
        self.resets = 0

    def step(self):
        """One Lloyd iteration; returns the assignment's counters plus the
        update's device time. A converged run restarts from the seeds."""
        g = self.g
        if self.converged:
            g.reseed(self.ini)
            self.converged = False
            self.resets += 1
        n = g.assign()
        st = g.stats()
        rec = dict(st)
        if st["iter"] > 1 and n == 0:
            self.converged = True
            rec["ms_update"] = 0.0
        else:
            g.update()
            su = g.stats()
            rec["ms_update"] = su["ms_update"]
            rec["centroid_nnz"] = su["centroid_nnz"]
        return rec

    def close(self):
        self.g.close()


def timed_window(path, args, stream, world, sampler=None):
    import torch
    for _ in range(args.warmup):
        path.step()
    if sampler:
        sampler.start()
    barrier_and_sync(world)
    l0 = path.g.stats()["launches"]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    per = [path.step() for _ in range(args.steps)]
    ev1.record(stream)
    barrier_and_sync(world)
    clocks = sampler.stop() if sampler else None
    launches = path.g.stats()["launches"] - l0 if path.resets == 0 else None
    return ev0.elapsed_time(ev1), per, launches, clocks


def roofline(per, w, nnz, prec, peaks, hbm_peak, sparse_file_bytes, dense_bytes):
    """Roofline of the assignment kernel over a window of iterations.

    Algorithmic bytes per launch: object CSR (nnz * 8 + (N + 1) * 8), per-object
    state (N * 16: labels old/new, own score read/write) and lambda (k), the
    sparse postings visited * bytes per posting and the dense-row entries read
    * bytes per entry. Each part is assigned to the memory that serves it: the
    CSR and the per-object state stream from HBM; postings and dense rows come
    from L2 when their structure fits in L2, else from HBM. The bound is the
    side that serves most of the bytes, and frac is achieved / that side's
    measured peak. A rate above the HBM peak can only come from L2, so it is
    labelled l2 whatever the structure sizes."""
    b_post = (B_POST16 if w.k <= 65536 else B_POST32)[prec]
    b_dense = B_DENSE[prec]
    fixed = nnz * 8 + (w.N + 1) * 8 + w.N * 16 + w.k
    ms = sum(p["ms_assign"] for p in per)
    sparse = sum(p["postings"] - p.get("dense_postings", 0) for p in per) * b_post
    dense = sum(p.get("dense_entries", 0) for p in per) * b_dense
    alg = fixed * len(per) + sparse + dense
    from_l2 = (sparse if sparse_file_bytes <= L2_BYTES else 0) + (dense if dense_bytes <= L2_BYTES else 0)
    achieved = alg / (ms / 1e3) / 1e9
    # a structure larger than L2 is still mostly served by L2 when its hot
    # lists fit there: a rate above the HBM peak shows that
    bound = "l2" if from_l2 > alg / 2 or achieved > hbm_peak else "hbm"
    peak = peaks["l2"] if bound == "l2" else hbm_peak
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": ("measured here: streaming reads of a 64 MB L2-resident buffer (CUDA events)"
                            if bound == "l2" else "MEASURED_PEAKS.json hbm_gbs (measured)"),
            "hbm_frac": achieved / hbm_peak, "l2_frac": achieved / peaks["l2"],
            "kernel": "assign_kernel", "bytes_per_launch": alg / len(per),
            "bytes_model": f"nnz*8 + (N+1)*8 + N*16 + k + postings read one by one*{b_post} B + dense-row "
                           f"entries read*{b_dense} B (no cache credit)",
            "bytes_from_l2_structures": from_l2 / max(alg, 1),
            "ms_assign_per_iter": ms / len(per),
            "ms_update_per_iter": sum(p["ms_update"] for p in per) / len(per),
            "postings_per_s": sum(p["postings"] for p in per) / (ms / 1e3),
            "dense_entries_per_s": sum(p.get("dense_entries", 0) for p in per) / (ms / 1e3),
            "simcalc_ratio": sum(p["simcalc"] for p in per) / (float(w.N) * w.k * len(per))}


def file_bytes(g, prec, k):
    """Bytes of the sparse scan copy (at most every posting of the file) and of
    the dense head rows of the current inverted file (library counters)."""
    st = g.stats()
    b_post = (B_POST16 if k <= 65536 else B_POST32)[prec]
    return st["centroid_nnz"] * b_post, st["dense_row_entries"] * B_DENSE[prec]


def trajectory(per):
    """The method-level counts of each iteration (independent of the posting
    precision and of which lists are held in dense rows)."""
    return [(int(p["changed"]), int(p["postings"]), int(p["filtered"]), int(p["simcalc"]), int(p["n_moving"]))
            for p in per]


def run_e2e(c, csr, w, ini, prec, args, stream, world, local):
    """The same window through the C ABI with host buffers. Every timed step
    takes its CSR from pinned host memory, runs one Lloyd iteration and reads
    the labels back. The host-to-device copy of step i+1's CSR runs on a copy
    stream into a device staging copy while step i computes (the context's
    CSR buffers are in use then); step i+1 starts with a device-to-device
    copy from the staging copy into the buffers the context reads. The first
    step's host copy is not overlapped, and every copy lies inside the timed
    region."""
    import torch
    from paper_2103_16141_gb300 import sivf as S
    rp_d, ix_d, vl_d = csr
    host = [torch.from_numpy(a).pin_memory() for a in (c.row_ptr, c.idx, c.val)]
    stage = [torch.empty_like(d) for d in csr]
    lab_h = torch.empty(w.N, dtype=torch.int32).pin_memory()
    copy_stream = torch.cuda.Stream()
    h2d_done, stage_free = torch.cuda.Event(), torch.cuda.Event()

    def h2d():
        with torch.cuda.stream(copy_stream):
            for st, h in zip(stage, host):
                st.copy_(h, non_blocking=True)
            h2d_done.record(copy_stream)

    path = Path(c, csr, w, ini, prec, args)
    try:
        for _ in range(args.warmup):
            path.step()
        E = args.e2e_steps if args.e2e_steps > 0 else args.steps
        sampler = ClockSampler(local)
        sampler.start()
        barrier_and_sync(world)
        t0 = time.perf_counter()
        h2d()
        with torch.cuda.stream(stream):
            for i in range(E):
                stream.wait_event(h2d_done)
                for d, st in zip(csr, stage):
                    d.copy_(st, non_blocking=True)
                stage_free.record(stream)
                if i + 1 < E:
                    copy_stream.wait_event(stage_free)
                    h2d()
                path.step()
                S.sivf_get_labels(path.g.ctx, lab_h.data_ptr(), False)
        barrier_and_sync(world)
        dt = max_over_ranks(time.perf_counter() - t0, world)
        clocks = sampler.stop()
    finally:
        path.close()
    h2d_bytes = sum(h.numel() * h.element_size() for h in host)
    return {"value": sum_over_ranks(float(w.N * E), world) / dt, "unit": "objects/s", "h2d_bytes_per_step": h2d_bytes,
            "d2h_bytes_per_step": w.N * 4, "steps": E, "clocks": clocks,
            "copies": "host CSR -> device staging copy on a copy stream, overlapping the previous step; "
                      "staging -> the context's CSR buffers at the step's start; labels -> pinned host",
            "window": f"iterations {args.warmup + 1}-{args.warmup + E}, a separate run from the same seeds"
                      + (" (the timed window)" if E == args.steps else "")}


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
    # after the timed region: one host-stepped run (one iteration per call, a
    # second context without the graph loop, whose device timers see every
    # step) for the device time of each iteration's assignment and update, and
    # the number of instances that have converged (no label changed)
    b.close()
    b = SIVFBatch(cs, [w.k for w in ws], inis, precision=prec, icp=args.icp, threads=args.threads,
                  ctas_per_sm=args.ctas_per_sm, use_graph=False, autotune=bool(args.autotune))
    per_ms = {"assign": [], "update": [], "instances_converged": []}
    for r in range(1, max_iter + 1):
        b.run(1)
        st1 = b.stats()
        conv = sum(b.instance_stats(m)["changed"] == 0 for m in range(len(ws))) if r > 1 else 0
        per_ms["assign"].append(round(st1["ms_assign"], 3))
        per_ms["update"].append(round(st1["ms_update"], 3) if conv < len(ws) else 0.0)
        per_ms["instances_converged"].append(int(conv))
        if conv == len(ws):
            break
    if rank == 0:
        nnz = sum(c.nnz for c in cs)
        line = {"metric": "objects/s (Lloyd iterations of SIVF spherical k-means, 64 batched instances)",
                "value": value, "unit": "objects/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": f"{prec}-postings/f32-products/fixed-point-sum", "data": "synthetic",
                "config": {"workload": f"c4: 64 instances, N={sum(w.N for w in ws)} total, nnz={nnz}, "
                                       f"k={sum(w.k for w in ws)} total, max k={max(w.k for w in ws)}",
                           "iterations_per_instance": [int(i) for i in its], "max_iter": max_iter},
                "per_iteration_ms": dict(per_ms, note="a host-stepped run after the timed region; the update "
                                                      "rewrites every instance's rows, converged ones included"),
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
    prec = args.precision or w.precision
    if args.impl == "reference":
        run_reference(args, w)
        return

    import torch
    from paper_2103_16141_gb300 import sivf as S

    world, rank, local = dist_setup(args.gpus)
    S.load()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    # each rank is an independent replica of the workload (the path needs no exchange)
    c = generate(w.N, w.D, w.zipf_s, w.mu, w.sigma, w.lo, w.hi, w.seed)
    ini = init_ids(w.N, w.k, w.init_seed)
    csr = (torch.from_numpy(c.row_ptr).to(dev), torch.from_numpy(c.idx).to(dev), torch.from_numpy(c.val).to(dev))
    hbm_peak, _ = load_peaks()
    peaks = measure_peaks(dev, stream)

    # the path of record
    path = Path(c, csr, w, ini, prec, args)
    sampler = ClockSampler(local)
    ms, per, launches, clocks = timed_window(path, args, stream, world, sampler)
    sparse_b, dense_b = file_bytes(path.g, prec, w.k)
    st_end = path.g.stats()
    lab_end = path.g.labels()
    path.close()
    value, ms_max = replica_throughput(w.N * args.steps, ms, world)
    roof = roofline(per, w, c.nnz, prec, peaks, hbm_peak, sparse_b, dense_b)
    trec = recorded_traffic(w, prec)
    roof["traffic"] = trec["dram_bytes_per_launch"] if trec else None
    roof["traffic_launch"] = trec.get("launch") if trec else None
    # the captured launch's own algorithmic bytes: traffic compares with this,
    # not with the window's mean bytes_per_launch (the iterations differ)
    roof["traffic_launch_algorithmic_bytes"] = trec.get("algorithmic_bytes_per_launch") if trec else None

    # the FP32 path on the same window
    vs_fp32 = None
    if not args.no_fp32 and prec != "fp32":
        p32 = Path(c, csr, w, ini, "fp32", args)
        ms32, per32, _, clocks32 = timed_window(p32, args, stream, world, ClockSampler(local))
        sb32, db32 = file_bytes(p32.g, "fp32", w.k)
        lab32 = p32.g.labels()
        p32.close()
        _, ms32_max = replica_throughput(w.N * args.steps, ms32, world)
        same_counts = trajectory(per) == trajectory(per32)
        same_labels = bool(np.array_equal(lab_end, lab32))
        vs_fp32 = {"sec_per_iter": ms_max / 1e3 / args.steps, "fp32_sec_per_iter": ms32_max / 1e3 / args.steps,
                   "speedup": ms32_max / ms_max, "precision": prec,
                   "fp32_roofline": roofline(per32, w, c.nnz, "fp32", peaks, hbm_peak, sb32, db32),
                   "same_counts_every_iteration": same_counts, "same_final_labels": same_labels,
                   "fp32_clocks": clocks32,
                   "equal_accuracy": "both paths re-score every object whose top-2 margin lies inside their "
                                     "derived error bound exactly (FP64 from the FP32 master centroids), so both "
                                     "give the argmax of the exact scores: the changed, posting, filtered, "
                                     "similarity and moving counts of every iteration and the labels after the "
                                     "window are compared"}

    e2e = None if args.no_e2e else run_e2e(c, csr, w, ini, prec, args, stream, world, local)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, c, ini, args.icp)

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": value, "unit": "objects/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == "fp32" else f"{prec}-postings/f32-products/fixed-point-sum",
            "data": "synthetic",
            "config": shared_config(w, c.nnz, args),
            "details": {"precision": prec, "icp": ICP_NAMES[args.icp], "sec_per_iter": ms_max / 1e3 / args.steps,
                        "parallelism": "replicas" if world > 1 else "single GPU",
                        "autotune": bool(args.autotune), "assign_threads": st_end["assign_threads"],
                        "score_buffer": "global" if st_end["assign_global"] else "shared",
                        "restarts_in_window": path.resets, "measured_peaks_gbs": peaks,
                        "dense_terms": st_end["dense_terms"], "dense_row_bytes": dense_b},
            "roofline": roof,
            "per_iteration": {"iteration": [int(p["iter"]) for p in per],
                              "postings": [int(p["postings"]) for p in per],
                              "dense_postings": [int(p.get("dense_postings", 0)) for p in per],
                              "dense_entries": [int(p.get("dense_entries", 0)) for p in per],
                              "filtered": [int(p["filtered"]) for p in per],
                              "rescored": [int(p["rescored"]) for p in per],
                              "changed": [int(p["changed"]) for p in per],
                              "n_moving_prev": [int(p["n_moving_prev"]) for p in per],
                              "ms_assign": [round(p["ms_assign"], 3) for p in per],
                              "ms_update": [round(p["ms_update"], 3) for p in per]},
            "gpu_launches": int(launches) if launches is not None else None,
            "clocks": clocks,
        }
        if vs_fp32:
            line["vs_fp32"] = vs_fp32
        if e2e:
            line["e2e"] = e2e
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
