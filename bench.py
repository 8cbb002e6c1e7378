#!/usr/bin/env python
"""Throughput of Local NBNN classification (Alg. 2) on the synthetic 256-class
index: 11.52M reference descriptors (256 classes x 30 images x 1,500), 500
query images x 1,500 descriptors, k = 10.

One step = one lnbnn_classify call over the whole batch (query preparation,
the tensor-core k+1 nearest-neighbour search, the class update and the
per-image argmin), with the index and the queries resident in HBM.  Prints one
JSON line (rank 0).  ``--impl reference`` times the CPU oracle instead, on a
bounded sample of the same workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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
sys.path.insert(0, ROOT)

from paper_1112_0059_gb300 import synth  # noqa: E402

METRIC = "query descriptors/s & images/s, 256-class index; tensor-pipe % of peak; serve p50/p99"
UNIT = "query descriptors/s"
KERNEL_SOURCES = ["paper_1112_0059_gb300/csrc/knn_tc.cu", "paper_1112_0059_gb300/csrc/sm103.cuh",
                  "paper_1112_0059_gb300/csrc/topk.cuh", "paper_1112_0059_gb300/csrc/knn_tc.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "knn_tc_traffic.json")


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="caltech256-like")
    p.add_argument("--k", type=int, default=10)
    p.add_argument("--classes", type=int, default=None, help="use the first C classes of the workload")
    p.add_argument("--query-images", type=int, default=None, help="use the first Q query images")
    p.add_argument("--method", choices=["local", "nbnn"], default="local",
                   help="local: Local NBNN (Alg. 2); nbnn: original NBNN (Alg. 1)")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--serve-rates", default="100,300,1000",
                   help="Poisson arrival rates (images/s) of the serving runs; empty to skip them")
    p.add_argument("--serve-seconds", type=float, default=2.5, help="arrival window of each serving run")
    return p.parse_args()


def workload_config(w: synth.Workload, k: int, method: str = "local") -> dict:
    local = method == "local"
    op_gb = w.n_ref * (128 + 16) * 2 / 1e9
    return {
        "workload": f"{w.name}: {w.notes}" + (f", k={k}" if local else "")
                    + (f"; first {w.n_classes} classes" if w.name.endswith(f"-C{w.n_classes}") else ""),
        "n_ref": w.n_ref,
        "n_classes": w.n_classes,
        "n_query_images": w.n_query_imgs,
        "query_descriptors": int(synth.query_counts(w).sum()),
        "k": k if local else None,
        "method": "Local NBNN (Alg. 2), exact search" if local else "original NBNN (Alg. 1), exact search",
        "l2": f"inputs larger than L2 ({op_gb:.2f} GB BF16 reference operand, re-read per query tile)",
        "seed": w.seed,
    }


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while running."""

    FIELDS = ["index", "clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, gpu_id: str | None):
        self.rows = []
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={','.join(self.FIELDS)}", "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == len(self.FIELDS):
                self.rows.append(parts)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            for n, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        pw = [float(r[3]) for r in self.rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.rows),
                "power_w_median": statistics.median(pw) if pw else None}


# ------------------------------------------------------------------ CPU oracle timing

def oracle_run(method, ref, labels, C, q, k, threads):
    import oracle
    off = np.array([0, len(q)])
    if method == "local":
        return oracle.local_nbnn(ref, labels, C, q, off, k, threads=threads)
    return oracle.nbnn(ref, labels, C, q, off, threads=threads)


def time_oracle(method, ref, labels, C, q, k, target_s: float, max_desc: int) -> dict:
    """The oracle on the first S query descriptors, S sized to about target_s
    seconds of this host's cores."""
    threads = os.cpu_count() or 1
    s = min(max_desc, max(threads, 8))
    t0 = time.perf_counter()
    oracle_run(method, ref, labels, C, q[:s], k, threads)
    dt = time.perf_counter() - t0
    per = dt / s
    s2 = int(min(max_desc, max(s, target_s / max(per, 1e-9))))
    s2 = max(threads, (s2 // threads) * threads) if s2 >= threads else s2
    if s2 > s:
        t0 = time.perf_counter()
        oracle_run(method, ref, labels, C, q[:s2], k, threads)
        dt = time.perf_counter() - t0
        s = s2
    name = f"Local NBNN, k={k}" if method == "local" else "original NBNN"
    return {"value": s / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"first {s} query descriptors of image 0 against all {len(ref)} references "
                      f"({name}), {dt:.1f} s"}


# ------------------------------------------------------------------ helpers

def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks() -> tuple[dict, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def traffic_per_launch(n_query_rows: int) -> float | None:
    """DRAM bytes per launch of the search kernel from a committed ncu capture,
    scaled to this launch by query rows; None if the kernel changed since."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    with open(TRAFFIC_FILE) as f:
        t = json.load(f)
    if t.get("kernel_hash") != kernel_hash():
        return None
    return t["dram_bytes_per_launch"] * n_query_rows / t["query_rows"]


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------ arms

def run_reference(args, w):
    world, rank, _ = dist_init()
    if rank != 0:
        return
    ref, labels = synth.reference_set(w)
    q, off, _ = synth.query_set(w)
    threads = os.cpu_count() or 1
    # per-step sample: sized from a calibration so the whole run stays within minutes
    cal = time_oracle(args.method, ref, labels, w.n_classes, q, args.k, target_s=min(args.cpu_seconds, 8.0),
                      max_desc=int(off[1]))
    s = max(1, int(round(cal["value"] * 6.0)))  # about 6 s per step
    s = min(s, int(off[1]))
    for _ in range(args.warmup):
        oracle_run(args.method, ref, labels, w.n_classes, q[:s], args.k, threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle_run(args.method, ref, labels, w.n_classes, q[:s], args.k, threads)
    dt = time.perf_counter() - t0
    value = s * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": workload_config(w, args.k, args.method),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"each step: first {s} query descriptors of image 0 against all {len(ref)} "
                                   f"references ({'Local NBNN, k=%d' % args.k if args.method == 'local' else 'original NBNN'}),"
                                   f" plain C oracle"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, w):
    import torch
    world, rank, local = dist_init()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else torch.cuda.current_device())
    from paper_1112_0059_gb300 import lnbnn
    lnbnn.load_library()

    ref, labels = synth.reference_set(w)
    q, off, _ = synth.query_set(w)
    M, n_img = int(q.shape[0]), int(off.shape[0] - 1)
    k = args.k
    ref_d = torch.from_numpy(ref).to(dev)
    lab_d = torch.from_numpy(labels).to(dev)
    q_d = torch.from_numpy(q).to(dev)
    off_d = torch.from_numpy(off).to(dev)
    index = lnbnn.Index(ref_d, lab_d, w.n_classes)
    del ref_d, lab_d
    totals = torch.empty((n_img, w.n_classes), dtype=torch.int64, device=dev)
    classes = torch.empty((n_img,), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    local = args.method == "local"

    def step():
        if local:
            index.lnbnn_classify(q_d, off_d, k, out=(totals, classes))
        else:
            index.nbnn_classify(q_d, off_d, out=(totals, classes))

    for _ in range(args.warmup):
        step()
    index.sync()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    gpu_uuid = None
    try:
        gpu_uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    index.profile_enable(True)
    barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(gpu_uuid)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clk = clocks.stop()
    index.sync()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    prof = index.profile_read()
    index.profile_enable(False)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([elapsed], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed = float(t.item())

    value = M * args.steps * world / elapsed
    peaks, peak_src = measured_peaks()
    search_ms = prof["search_ms"] / max(prof["search_launches"], 1)
    flops = 2.0 * 128 * w.n_ref * M  # algorithmic, per launch
    achieved = flops / (search_ms / 1e3) / 1e12
    # both methods run the same tensor-core scan (K = 128 + a 16-wide extension);
    # the roofline counts the algorithmic 2 * 128 flops per (query, reference) pair
    roofline = {"bound": "tensor", "achieved": achieved, "peak": float(peaks["bf16_tflops_sustained"]),
                "unit": "TFLOP/s", "traffic": traffic_per_launch(M) if local else None,
                "kernel": "tc_scan_kernel<KnnEpilogue<16>>" if local else "tc_scan_kernel<NbnnEpilogue>",
                "peak_source": f"bf16_tflops_sustained ({peak_src})"}
    roofline.update({"frac": roofline["achieved"] / roofline["peak"], "flops_per_launch": flops,
                     "avg_launch_ms": search_ms})

    e2e = None
    if not args.no_e2e:
        q_h = torch.from_numpy(q).pin_memory()
        off_h = torch.from_numpy(off).pin_memory()
        tot_h = torch.empty((n_img, w.n_classes), dtype=torch.int64).pin_memory()
        cls_h = torch.empty((n_img,), dtype=torch.int32).pin_memory()
        qn, on, tn, cn = q_h.numpy(), off_h.numpy(), tot_h.numpy(), cls_h.numpy()
        hk = k if local else None
        index.classify_host(qn, on, hk, tn, cn)  # warm the staging buffer
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            index.classify_host(qn, on, hk, tn, cn)
        e2e_dt = time.perf_counter() - t0
        if world > 1:
            import torch.distributed as dist
            t = torch.tensor([e2e_dt], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_dt = float(t.item())
        e2e = {"value": M * args.steps * world / e2e_dt, "unit": UNIT, "h2d_bytes_per_step": int(q.nbytes + off.nbytes),
               "d2h_bytes_per_step": int(tn.nbytes + cn.nbytes),
               "api": ("lnbnn" if local else "nbnn") + "_classify_host (pinned host buffers; copies, classify, "
                      "copy-back, sync per step)"}

    serve_block = None
    rates = [float(r) for r in args.serve_rates.split(",") if r.strip()]
    if rates and args.method == "local" and w.n_classes == synth.workload("serving").n_classes:
        serve_block = run_serving(index, rates, args.serve_seconds, k)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = time_oracle(args.method, ref, labels, w.n_classes, q, k, args.cpu_seconds, int(off[1]))

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": workload_config(w, k, args.method),
            "images_per_s": n_img * args.steps * world / elapsed,
            "roofline": roofline,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "serve": serve_block,
            "gpu_launches": int(prof["kernel_launches"]),
            "clocks": clk,
            "profile": {"search_ms_total": prof["search_ms"], "other_ms_total": prof["other_ms"],
                        "calls": prof["calls"], "search_sm_clock_ghz": prof["search_sm_clock_ghz"],
                        "search_cycles_per_tile": prof["search_cycles_per_tile"],
                        "mma_cycles_per_tile": 9 * 128},
        }
        print(json.dumps(line), flush=True)
    index.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_serving(index, rates, seconds, k) -> dict:
    """The continuous-batching server over the resident index: Poisson
    arrivals of query images with log-uniform [100, 4000] descriptors."""
    from paper_1112_0059_gb300 import serve
    w = synth.workload("serving")
    cfg = {"slots": 3, "max_batch_queries": 16384, "max_batch_images": 256, "graphs": True, "graph_granule": 2048}
    runs, first = [], 0
    with serve.Server(index, k=k, method="local", **cfg) as srv:
        srv.run(serve.poisson_requests(w, 1000.0, 8, seed=99, first_image=100000))  # warm-up
        for rate in rates:
            n = max(8, int(rate * seconds))
            reqs = serve.poisson_requests(w, rate, n, seed=0, first_image=first)
            first += n
            srv.log = []
            done = srv.run(reqs)
            st = serve.latency_stats(done, srv.log)
            st["rate_offered"] = rate
            runs.append(st)
    return {"form": "exact", "k": k, "workload": "256-class index; Poisson arrivals; log-uniform [100, 4000] "
            "descriptors per image; latency = arrival to totals and class on the host", **cfg, "runs": runs}


def main():
    args = parse_args()
    w = synth.workload(args.workload)
    if args.classes:
        w = w.with_classes(args.classes)
    if args.query_images:
        w = w.with_query_imgs(args.query_images)
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
