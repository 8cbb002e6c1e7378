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

# Measurements reported beside the headline, each a block of the JSON line.
SECTIONS = {
    "uneven": "1,024 query images of U{200..3000} descriptors in one call on the 256-class index: exact and the "
              "FP8 shortlist at m = 24, 32, 64, 128, with recall, score error and class agreement",
    "kc": "Local NBNN at k = 1, 10, 50, 100 and original NBNN on the first 32 and all 256 classes "
          "(100 query images): run time against k and class count",
    "caltech101": "the 101-class index (1.515M references, 200 images x 1,000 descriptors): Local NBNN at "
                  "k = 1, 10, 50 against original NBNN",
    "serve": "the continuous-batching server: Poisson arrivals, p50/p99 latency, exact and FP8",
    "single": "one query image of 100 / 632 / 1,000 / 4,000 descriptors at a time, k = 10, 50, 100, exact and FP8 "
              "(shortlist 24, 64, 128)",
    "logodds": "NBNN as a sum of log-odds increments (all or only the positive ones) for several beta",
}
DEFAULT_SECTIONS = "uneven,kc,caltech101,serve"


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
    p.add_argument("--shortlist", type=int, default=None,
                   help="time the FP8 E4M3 shortlist search (shortlist length m) instead of the exact one")
    p.add_argument("--fp8-shortlist", type=int, default=24,
                   help="shortlist of the FP8 block and FP8 serving runs reported beside the exact form (0: skip)")
    p.add_argument("--serve-rates", default="100,300,1000",
                   help="Poisson arrival rates (images/s) of the serving runs; empty to skip them")
    p.add_argument("--serve-seconds", type=float, default=2.5, help="arrival window of each serving run")
    p.add_argument("--sections", default=DEFAULT_SECTIONS,
                   help="measurements reported beside the headline (comma-separated; empty for none): "
                        + ", ".join(f"{k} ({v})" for k, v in SECTIONS.items()))
    p.add_argument("--schedule", default="",
                   help="fixed launch schedule of the scans, e.g. 'query_tiles=2,persistent=1,splits=19' "
                        "(lnbnn_set_schedule; results never change); empty: automatic")
    p.add_argument("--recall-rows", type=int, default=8192,
                   help="seeded random query rows (all images) of the FP8 recall against the exact search")
    p.add_argument("--oracle-recall-rows", type=int, default=256,
                   help="seeded random query rows of the FP8 recall against the CPU oracle (0: skip)")
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


def _traffic_entry(kernel: str) -> dict | None:
    if not os.path.exists(TRAFFIC_FILE):
        return None
    with open(TRAFFIC_FILE) as f:
        t = json.load(f)
    if t.get("kernel_hash") != kernel_hash() or kernel not in t.get("kernels", {}):
        return None
    return t["kernels"][kernel]


def traffic_per_launch(kernel: str, n_query_rows: int, n_ref: int) -> float | None:
    """DRAM bytes of one launch of a search kernel from a committed ncu capture:
    the capture's own figure for a launch of the same size, else scaled by
    query rows x references (from a smaller case an upper bound: a larger
    launch reuses L2 more); None if the kernel changed since or was not
    captured."""
    k = _traffic_entry(kernel)
    if k is None:
        return None
    return k["dram_bytes"] * (n_query_rows * n_ref) / (k["query_rows"] * k["n_ref"])


def traffic_note(kernel: str, n_query_rows: int, n_ref: int) -> str:
    """Where roofline.traffic comes from."""
    k = _traffic_entry(kernel)
    if k is None:
        return "no ncu capture of the current kernel sources"
    if (k["query_rows"], k["n_ref"]) == (n_query_rows, n_ref):
        return ("ncu one-pass capture of this launch (dram__bytes_read.sum + dram__bytes_write.sum); "
                "profiles/knn_tc_traffic.json")
    return (f"ncu DRAM bytes of a launch of {k['query_rows']:,} query rows x {k['n_ref']:,} references scaled by "
            "query rows x references; profiles/knn_tc_traffic.json")


def max_over_ranks(x: float, device=None) -> float:
    """The largest value of x over all ranks (x itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


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
    world, rank, local_rank = dist_init()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank if world > 1 else torch.cuda.current_device())
    from paper_1112_0059_gb300 import lnbnn
    lnbnn.load_library()

    ref, labels = synth.reference_set(w)
    q, off, _ = synth.query_set(w)
    M, n_img = int(q.shape[0]), int(off.shape[0] - 1)
    k = args.k
    local = args.method == "local"
    shortlist = args.shortlist if local else None  # the timed form: exact, or the FP8 shortlist search
    fp8_m = args.fp8_shortlist if local and not shortlist else 0  # FP8 form reported beside the exact one
    ref_d = torch.from_numpy(ref).to(dev)
    lab_d = torch.from_numpy(labels).to(dev)
    q_d = torch.from_numpy(q).to(dev)
    off_d = torch.from_numpy(off).to(dev)
    index = lnbnn.Index(ref_d, lab_d, w.n_classes)
    del ref_d, lab_d
    if args.schedule:
        index.set_schedule(**{k.strip(): int(v) for k, v in (kv.split("=") for kv in args.schedule.split(","))})
    if shortlist or fp8_m:
        index.prepare_fp8()
    totals = torch.empty((n_img, w.n_classes), dtype=torch.int64, device=dev)
    classes = torch.empty((n_img,), dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def make_step(m_short, out):
        def step():
            if local:
                index.lnbnn_classify(q_d, off_d, k, out=out, shortlist=m_short)
            else:
                index.nbnn_classify(q_d, off_d, out=out)
        return step

    step = make_step(shortlist, (totals, classes))
    for _ in range(args.warmup):
        step()
    index.sync()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(fn, steps):
        """Device time of `steps` calls of fn (CUDA events on the launching stream) and the call profile."""
        index.profile_enable(True)
        barrier()
        torch.cuda.synchronize(dev)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(steps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        index.sync()
        prof = index.profile_read()
        index.profile_enable(False)
        return max_over_ranks(ev0.elapsed_time(ev1) / 1e3, dev), prof

    gpu_uuid = None
    try:
        gpu_uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(gpu_uuid)
    elapsed, prof = timed(step, args.steps)
    clk = clocks.stop()

    value = M * args.steps * world / elapsed
    peaks, peak_src = measured_peaks()
    plan = index.plan_search(M, (shortlist or k + 1) if local else 1, fp8=bool(shortlist)) if local else None
    roofline = scan_roofline(prof, w.n_ref, M, peaks, peak_src, local, shortlist, k, plan)
    if plan:
        roofline["schedule"] = plan
    roofline["traffic"] = traffic_per_launch(roofline["kernel"], M, w.n_ref)
    roofline["traffic_note"] = traffic_note(roofline["kernel"], M, w.n_ref)

    e2e = None
    if not args.no_e2e:
        q_h = torch.from_numpy(q).pin_memory()
        off_h = torch.from_numpy(off).pin_memory()
        tot_h = torch.empty((n_img, w.n_classes), dtype=torch.int64).pin_memory()
        cls_h = torch.empty((n_img,), dtype=torch.int32).pin_memory()
        qn, on, tn, cn = q_h.numpy(), off_h.numpy(), tot_h.numpy(), cls_h.numpy()
        hk = k if local else None
        index.classify_host(qn, on, hk, tn, cn, shortlist=shortlist)  # warm the staging buffer
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            index.classify_host(qn, on, hk, tn, cn, shortlist=shortlist)
        e2e_dt = max_over_ranks(time.perf_counter() - t0, dev)
        api = "lnbnn_classify_fp8_host" if shortlist else ("lnbnn" if local else "nbnn") + "_classify_host"
        e2e = {"value": M * args.steps * world / e2e_dt, "unit": UNIT, "h2d_bytes_per_step": int(q.nbytes + off.nbytes),
               "d2h_bytes_per_step": int(tn.nbytes + cn.nbytes),
               "api": api + " (pinned host buffers; copies, classify, copy-back, sync per step)"}

    # accuracy of the FP8 form against the exact search (parity-tested against the oracle)
    fp8_block = None
    if local and (shortlist or fp8_m):
        m_short = shortlist or fp8_m
        t_x = torch.empty_like(totals)
        c_x = torch.empty_like(classes)
        t_f = torch.empty_like(totals)
        c_f = torch.empty_like(classes)
        make_step(None, (t_x, c_x))()
        fp8_step = make_step(m_short, (t_f, c_f))
        if shortlist:
            fp8_step()
            fp8_block = {"shortlist": m_short}
        else:
            for _ in range(args.warmup):
                fp8_step()
            el8, prof8 = timed(fp8_step, args.steps)
            fp8_block = {"shortlist": m_short, "value": M * args.steps * world / el8, "unit": UNIT,
                         "images_per_s": n_img * args.steps * world / el8, "ms_per_step": el8 / args.steps * 1e3,
                         "roofline": scan_roofline(prof8, w.n_ref, M, peaks, peak_src, True, m_short, k,
                                                   index.plan_search(M, m_short, fp8=True)),
                         "gpu_launches": int(prof8["kernel_launches"])}
            fp8_block["roofline"]["traffic"] = traffic_per_launch(fp8_block["roofline"]["kernel"], M, w.n_ref)
            fp8_block["roofline"]["traffic_note"] = traffic_note(fp8_block["roofline"]["kernel"], M, w.n_ref)
        index.sync()
        fp8_block.update(fp8_accuracy(index, q_d, q, ref, k, m_short, t_x, c_x, t_f, c_f, args.recall_rows,
                                      args.oracle_recall_rows if rank == 0 and world == 1 else 0))

    sections = [x for x in args.sections.split(",") if x.strip()]
    serve_block = None
    rates = [float(r) for r in args.serve_rates.split(",") if r.strip()]
    if "serve" in sections and rates and local and w.n_classes == synth.workload("serving").n_classes:
        cls_x, cls_f = {}, {}
        serve_block = {"exact": run_serving(index, rates, args.serve_seconds, k, None, cls_x)}
        if fp8_m or shortlist:
            serve_block["fp8"] = run_serving(index, rates, args.serve_seconds, k, shortlist or fp8_m, cls_f)
            # both forms served the same images (same seeds): their class decisions, image by image
            same = [cls_x[key] == cls_f[key] for key in cls_x if key in cls_f]
            serve_block["fp8_class_agreement_with_exact"] = {
                "images": len(same), "agreement": float(np.mean(same)) if same else None}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = time_oracle(args.method, ref, labels, w.n_classes, q, k, args.cpu_seconds, int(off[1]))

    extra = {}
    if rank == 0 and world == 1 and w.name == "caltech256-like" and local:
        extra = run_sections(sections, index, ref, labels, k, args.fp8_shortlist or 32)

    if rank == 0:
        cfg = workload_config(w, k, args.method)
        if shortlist:
            cfg["method"] = f"Local NBNN (Alg. 2), FP8 E4M3 shortlist search (m = {shortlist}) + exact rerank"
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "e4m3" if shortlist else "bf16", "data": "synthetic",
            "config": cfg,
            "images_per_s": n_img * args.steps * world / elapsed,
            "roofline": roofline,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "fp8": fp8_block,
            "serve": serve_block,
            **extra,
            "gpu_launches": int(prof["kernel_launches"]),
            "clocks": clk,
            "profile": {"search_ms_total": prof["search_ms"], "other_ms_total": prof["other_ms"],
                        "calls": prof["calls"], "search_sm_clock_ghz": prof["search_sm_clock_ghz"],
                        "search_cycles_per_tile": prof["search_cycles_per_tile"],
                        "mma_cycles_per_tile": 5 * 128 if shortlist else 9 * 128},
        }
        print(json.dumps(line), flush=True)
    index.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _sample(M: int, n: int, seed: int) -> np.ndarray:
    """n distinct seeded random rows of [0, M) (all rows if n >= M), sorted."""
    if n >= M:
        return np.arange(M)
    return np.sort(np.random.default_rng(seed).choice(M, size=n, replace=False))


def fp8_accuracy(index, q_d, q, ref, k, m, t_x, c_x, t_f, c_f, recall_rows, oracle_rows) -> dict:
    """Recall of the k+1 neighbours of the FP8 shortlist search on seeded
    random rows of all images, against the exact tensor-core search and (on
    fewer rows) against the CPU oracle directly; int64 score error and class
    agreement of the classify calls against the exact ones."""
    import torch
    M = int(q_d.shape[0])
    rows = _sample(M, recall_rows, 7)
    rd = torch.from_numpy(rows).to(q_d.device)
    qs = q_d.index_select(0, rd)
    i_x, _ = index.knn_search(qs, k + 1)
    i_f, _ = index.knn_search(qs, k + 1, shortlist=m)
    index.sync()
    ix_, if_ = i_x.cpu().numpy(), i_f.cpu().numpy()
    out = {"knn_recall": float(np.mean([len(set(a) & set(b)) for a, b in zip(ix_, if_)]) / (k + 1)),
           "recall_sample": f"{len(rows)} seeded random query rows of all images, the k+1 = {k + 1} neighbours, "
                            "against the exact tensor-core search"}
    if oracle_rows:
        import oracle
        orows = _sample(M, oracle_rows, 8)
        _, oj = oracle.knn(ref, q[orows], k + 1)
        od = torch.from_numpy(orows).to(q_d.device)
        j_f, _ = index.knn_search(q_d.index_select(0, od), k + 1, shortlist=m)
        index.sync()
        jf = j_f.cpu().numpy()
        out["knn_recall_vs_oracle"] = float(np.mean([len(set(a) & set(b)) for a, b in zip(oj, jf)]) / (k + 1))
        out["oracle_recall_sample"] = f"{len(orows)} seeded random query rows, against the CPU oracle's exact kNN"
    if t_x is not None:
        tx, tf = t_x.cpu().numpy(), t_f.cpu().numpy()
        out.update({"class_agreement": float((c_x.cpu().numpy() == c_f.cpu().numpy()).mean()),
                    "score_rel_error": float(np.abs(tf - tx).sum() / max(1, np.abs(tx).sum())),
                    "score_max_abs_error": int(np.abs(tf - tx).max()),
                    "reference": "the exact tensor-core search (bit-exact with the oracle in the parity tests)"})
    return out


def _timed(fn, reps: int, warm: int = 1) -> float:
    """Median device time (s) of reps calls after warm calls (CUDA events on
    the current stream, the queries already on the device)."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return statistics.median(times)


def section_uneven(index, ref, k, shortlists=(24, 32, 64, 128)) -> dict:
    """The batched uneven workload: 1,024 images of U{200..3000} descriptors,
    flattened with offsets, one classify call per form."""
    import torch
    w = synth.workload("batched-uneven")
    q, off, _ = synth.query_set(w)
    qd, od = torch.from_numpy(q).cuda(), torch.from_numpy(off).cuda()
    M, n_img = len(q), len(off) - 1
    res = {"workload": f"{w.name}: {w.notes}; {M:,} descriptors", "k": k, "runs": []}
    index.prepare_fp8()
    outs = {}
    for m in (None, *shortlists):
        tot = torch.empty((n_img, w.n_classes), dtype=torch.int64, device="cuda")
        cls = torch.empty((n_img,), dtype=torch.int32, device="cuda")
        t = _timed(lambda: index.lnbnn_classify(qd, od, k, out=(tot, cls), shortlist=m), 1)
        index.sync()
        outs[m] = (tot, cls)
        plan = index.plan_search(M, m if m else k + 1, fp8=m is not None)
        rec = {"form": "exact" if m is None else "fp8", "shortlist": m, "seconds": t, "desc_per_s": M / t,
               "images_per_s": n_img / t, "plan": plan}
        if m is not None:
            tx, cx = outs[None]
            rec.update(fp8_accuracy(index, qd, q, ref, k, m, tx, cx, tot, cls, 8192, 256 if m == shortlists[0] else 0))
        res["runs"].append(rec)
    return res


def section_kc(ref, labels, index, ks=(1, 10, 50, 100), classes=(32, 256), q_imgs=100) -> dict:
    """Run time against k and class count: the first C classes of the
    256-class index (N = C x 45,000), 100 query images."""
    import torch
    from paper_1112_0059_gb300 import lnbnn
    res = {"query_images": q_imgs, "runs": []}
    for C in classes:
        w = synth.workload("caltech256-like").with_classes(C).with_query_imgs(q_imgs)
        n = w.n_ref
        q, off, _ = synth.query_set(w)
        qd, od = torch.from_numpy(q).cuda(), torch.from_numpy(off).cuda()
        own = None
        if n == index.n_ref:
            ix = index
        else:
            own = ix = lnbnn.Index(torch.from_numpy(ref[:n]).cuda(), torch.from_numpy(labels[:n]).cuda(), C)
        try:
            for k in ks:
                t = _timed(lambda: ix.lnbnn_classify(qd, od, k), 2)
                res["runs"].append({"C": C, "n_ref": n, "method": "local", "k": k, "seconds": t,
                                    "desc_per_s": len(q) / t, "tflops": 2 * 128 * n * len(q) / t / 1e12})
            t = _timed(lambda: ix.nbnn_classify(qd, od), 2)
            res["runs"].append({"C": C, "n_ref": n, "method": "nbnn", "k": None, "seconds": t,
                                "desc_per_s": len(q) / t, "tflops": 2 * 128 * n * len(q) / t / 1e12})
            ix.sync()
        finally:
            if own is not None:
                own.close()
    return res


def section_caltech101(ks=(1, 10, 50)) -> dict:
    """The 101-class index: Local NBNN at several k against original NBNN."""
    import torch
    from paper_1112_0059_gb300 import lnbnn
    w = synth.workload("caltech101-like")
    ref, labels = synth.reference_set(w)
    q, off, _ = synth.query_set(w)
    qd, od = torch.from_numpy(q).cuda(), torch.from_numpy(off).cuda()
    res = {"workload": f"{w.name}: {w.notes}", "runs": []}
    with lnbnn.Index(torch.from_numpy(ref).cuda(), torch.from_numpy(labels).cuda(), w.n_classes) as ix:
        for k in ks:
            t = _timed(lambda: ix.lnbnn_classify(qd, od, k), 3)
            res["runs"].append({"method": "local", "k": k, "seconds": t, "desc_per_s": len(q) / t,
                                "images_per_s": (len(off) - 1) / t, "tflops": 2 * 128 * w.n_ref * len(q) / t / 1e12,
                                "plan": ix.plan_search(len(q), k + 1)})
        t = _timed(lambda: ix.nbnn_classify(qd, od), 3)
        res["runs"].append({"method": "nbnn", "k": None, "seconds": t, "desc_per_s": len(q) / t,
                            "images_per_s": (len(off) - 1) / t, "tflops": 2 * 128 * w.n_ref * len(q) / t / 1e12})
        ix.sync()
    return res


def section_single(index, sizes=(100, 632, 1000, 4000), ks=(10, 50, 100)) -> dict:
    """One query image at a time (few query tiles, many reference splits)."""
    import torch
    w = synth.workload("caltech256-like")
    res = {"runs": []}
    for n in sizes:
        qd = torch.from_numpy(synth.query_image(w, 7, n)).cuda()
        for k in ks:
            m = {10: 24, 50: 64, 100: 128}.get(k, 2 * (k + 1))  # k = 10: the FP8 form of the headline
            for form, sl in (("exact", None), ("fp8", m)):
                t = _timed(lambda: index.knn_search(qd, k + 1, shortlist=sl), 5)
                res["runs"].append({"descriptors": n, "k": k, "form": form, "shortlist": sl, "ms": t * 1e3,
                                    "plan": index.plan_search(n, sl or k + 1, fp8=sl is not None)})
    index.sync()
    return res


def section_logodds(index, betas=(1e-6, 1e-5, 1e-4, 1e-3), q_imgs=100) -> dict:
    """NBNN as a sum of log-odds increments (Section 3.1), all or positive only."""
    import torch
    w = synth.workload("caltech256-like").with_query_imgs(q_imgs)
    q, off, _ = synth.query_set(w)
    qd, od = torch.from_numpy(q).cuda(), torch.from_numpy(off).cuda()
    _, c_nbnn = index.nbnn_classify(qd, od)
    c_nbnn = c_nbnn.cpu().numpy()
    res = {"query_images": q_imgs, "runs": []}
    for beta in betas:
        for pos in (False, True):
            t = _timed(lambda: index.nbnn_logodds_classify(qd, od, beta, pos), 2)
            _, c, n = index.nbnn_logodds_classify(qd, od, beta, pos)
            index.sync()
            res["runs"].append({"beta": beta, "positive_only": pos, "seconds": t, "desc_per_s": len(q) / t,
                                "increments_per_desc": float(n.cpu().numpy().sum()) / len(q),
                                "agreement_with_nbnn": float((c.cpu().numpy() == c_nbnn).mean())})
    return res


def run_sections(sections, index, ref, labels, k, m) -> dict:
    """The requested sections (serving runs elsewhere), each timed outside the
    headline's timed region."""
    out = {}
    for name in sections:
        t0 = time.perf_counter()
        if name == "uneven":
            out[name] = section_uneven(index, ref, k)
        elif name == "kc":
            out[name] = section_kc(ref, labels, index)
        elif name == "caltech101":
            out[name] = section_caltech101()
        elif name == "single":
            out[name] = section_single(index)
        elif name == "logodds":
            out[name] = section_logodds(index)
        else:
            continue
        out[name]["about"] = SECTIONS[name]
        out[name]["wall_s"] = time.perf_counter() - t0
    return out


def list_kind(K1: int) -> int:
    """Register-list size the search kernel uses for lists of K1 (0: heap)."""
    return 16 if K1 <= 16 else 24 if K1 <= 24 else 32 if K1 <= 32 else 64 if K1 <= 64 else 0


def kernel_name(local: bool, shortlist, k: int, plan: dict | None = None) -> str:
    """The search kernel a launch runs: operand format, epilogue (list kind),
    query tiles per CTA and whether it claims reference chunks, as in the
    profiler's kernel names."""
    qt = (plan or {}).get("tile_m", 128) // 128
    claim = int((plan or {}).get("chunked", 0))
    if not local:
        return f"tc_scan_kernel<FmtBf16, NbnnEpilogue, {qt}, 0>"
    K1 = shortlist or k + 1
    fmt = "FmtE4m3" if shortlist else "FmtBf16"
    if plan and plan.get("list_storage") == "shared memory":
        epi = "KnnSmemEpilogue<64>"
    else:
        epi = f"KnnEpilogue<{list_kind(K1)}>"
    return f"tc_scan_kernel<{fmt}, {epi}, {qt}, {claim}>"


def scan_roofline(prof, n_ref, M, peaks, peak_src, local, shortlist, k: int = 10, plan: dict | None = None) -> dict:
    """Roofline of the search kernel from the call profile: algorithmic
    2 * 128 flops per (query, reference) pair over its mean launch time."""
    search_ms = prof["search_ms"] / max(prof["search_launches"], 1)
    flops = 2.0 * 128 * n_ref * M
    achieved = flops / (search_ms / 1e3) / 1e12
    if shortlist:
        # E4M3 contraction: twice the BF16 rate (nominal dense 4.5 vs 2.25 PFLOP/s)
        peak = 2.0 * float(peaks["bf16_tflops_sustained"])
        src = f"2 x bf16_tflops_sustained ({peak_src}), the nominal fp8/bf16 ratio"
    else:
        peak = float(peaks["bf16_tflops_sustained"])
        src = f"bf16_tflops_sustained ({peak_src})"
    kernel = kernel_name(local, shortlist, k, plan)
    out = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "traffic": None, "kernel": kernel, "peak_source": src, "flops_per_launch": flops,
           "avg_launch_ms": search_ms}
    clk = (peaks.get("clocks_under_load") or {}).get("sm_mhz_median")
    if clk:
        out["peak_sm_mhz"] = clk  # the SM clock the peak was measured at
    cpt = prof.get("search_cycles_per_tile") or 0.0
    if cpt > 0:
        # Clock-free view: SM cycles per 128 x 256 tile against the MMA floor
        # (BF16: 8 MMAs of K = 16 plus the K-extension, 9 x 128 cycles; E4M3:
        # 4 MMAs of K = 32 plus the BF16 extension, 5 x 128), and the share of
        # that floor which is algorithmic work (the extension's 16 of 144, or
        # 1 of 5 MMAs, is not).
        floor, algo = (5 * 128, 4 / 5) if shortlist else (9 * 128, 128 / 144)
        out.update({"kernel_sm_ghz": prof.get("search_sm_clock_ghz"), "cycles_per_tile": cpt,
                    "mma_floor_cycles_per_tile": floor, "tensor_pipe_frac_at_kernel_clock": floor / cpt,
                    "algorithmic_frac_at_kernel_clock": floor / cpt * algo})
    return out


def run_serving(index, rates, seconds, k, shortlist, classes_out: dict | None = None) -> dict:
    """The continuous-batching server over the resident index: Poisson
    arrivals of query images with log-uniform [100, 4000] descriptors.
    classes_out (optional) receives {(rate, request id): class} of every
    served image."""
    from paper_1112_0059_gb300 import serve
    w = synth.workload("serving")
    cfg = {"slots": 2, "max_batch_queries": 16384, "max_batch_images": 256, "graphs": True}
    runs, first = [], 0
    with serve.Server(index, k=k, method="local", shortlist=shortlist, **cfg) as srv:
        srv.run(serve.poisson_requests(w, 1000.0, 8, seed=99, first_image=100000))  # warm-up
        for rate in rates:
            n = max(8, int(rate * seconds))
            reqs = serve.poisson_requests(w, rate, n, seed=0, first_image=first)
            first += n
            srv.log = []
            done = srv.run(reqs)
            if classes_out is not None:
                classes_out.update({(rate, r.rid): r.cls for r in done})
            st = serve.latency_stats(done, srv.log)
            st["rate_offered"] = rate
            runs.append(st)
    form = "exact" if shortlist is None else f"FP8 E4M3 shortlist m = {shortlist} + exact rerank"
    return {"form": form, "k": k, "workload": "256-class index; Poisson arrivals; log-uniform [100, 4000] "
            "descriptors per image; latency = arrival to totals and class on the host", **cfg,
            "admission": f"arrival order into the next free slot while its batch stays within "
                         f"{cfg['max_batch_queries']:,} descriptors and {cfg['max_batch_images']} images; a request "
                         f"of more than {cfg['max_batch_queries']:,} descriptors is refused (ValueError)",
            "graph_buckets": f"{len(serve.graph_buckets(cfg['max_batch_queries']))} query-count buckets, "
                             "every multiple of 128 up to 4,096, then about 25% apart", "runs": runs}


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
