"""Measurement sweeps on the synthetic workloads (GPU, CUDA events).

    python -m paper_1112_0059_gb300.sweep [--parts kc,fp8,logodds,single,uneven] [--query-images Q] [--reps R]

kc      Local NBNN (Alg. 2) run time against k, on the first C classes of the
        256-class index (N = C x 45,000 references), with original NBNN
        (Alg. 1) beside it: how the cost grows with k and with the class count.
fp8     the FP8 E4M3 shortlist search at several shortlist lengths m against
        the exact search on the 256-class index: throughput, kNN recall of the
        k+1 neighbours, int64 score error and class agreement.
logodds NBNN as a sum of log-odds increments (Section 3.1) on the 256-class
        index for several kernel widths beta: run time, the share of device
        time outside the scan, the average number of increments added per
        descriptor (all, or only the positive ones: Table 1's measure) and the
        agreement of the chosen classes with NBNN's (Alg. 1).
single  one query image of 100 / 632 / 1,000 / 4,000 descriptors at a time (the serving
        regime: few query tiles, many reference splits) for k = 10, 50, 100, exact and
        with the FP8 shortlist (m = 32, 64, 128): device time per call.
uneven  1,024 query images with uniform [200, 3000] descriptors, flattened
        with offsets, one classify call, exact and FP8, before and after the
        split-schedule autotuner.

Every timing is the median of R calls after one warm-up, measured with CUDA
events on the launching stream; the index is resident and the queries are
on the device.  One JSON object per measurement goes to stdout, then a
markdown table per part.
"""
from __future__ import annotations

import argparse
import json
import statistics

import numpy as np

from . import lnbnn, synth


def _timed(fn, reps: int) -> float:
    import torch
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


def _emit(rows: list, rec: dict) -> None:
    rows.append(rec)
    print(json.dumps(rec), flush=True)


def part_kc(ref, labels, classes, ks, q_imgs, reps, rows):
    import torch
    for C in classes:
        w = synth.workload("caltech256-like").with_classes(C).with_query_imgs(q_imgs)
        n = C * w.ref_imgs_per_class * w.ref_desc_per_img
        q, off, _ = synth.query_set(w)
        qd, od = torch.from_numpy(q).cuda(), torch.from_numpy(off).cuda()
        with lnbnn.Index(torch.from_numpy(ref[:n]).cuda(), torch.from_numpy(labels[:n]).cuda(), C) as ix:
            for k in ks:
                t = _timed(lambda: ix.lnbnn_classify(qd, od, k), reps)
                ix.sync()
                _emit(rows, {"part": "kc", "method": "local", "C": C, "n_ref": n, "k": k, "queries": len(q),
                             "seconds": t, "desc_per_s": len(q) / t, "tflops": 2 * 128 * n * len(q) / t / 1e12})
            t = _timed(lambda: ix.nbnn_classify(qd, od), reps)
            ix.sync()
            _emit(rows, {"part": "kc", "method": "nbnn", "C": C, "n_ref": n, "k": None, "queries": len(q),
                         "seconds": t, "desc_per_s": len(q) / t, "tflops": 2 * 128 * n * len(q) / t / 1e12})


def _recall(ix, qd, k, m, sample):
    i_x, _ = ix.knn_search(qd[:sample], k + 1)
    i_f, _ = ix.knn_search(qd[:sample], k + 1, shortlist=m)
    ix.sync()
    a, b = i_x.cpu().numpy(), i_f.cpu().numpy()
    return float(np.mean([len(set(a[r]) & set(b[r])) for r in range(sample)]) / (k + 1))


def _accuracy(ix, qd, od, k, m, sample):
    t_x, c_x = ix.lnbnn_classify(qd, od, k)
    t_f, c_f = ix.lnbnn_classify(qd, od, k, shortlist=m)
    ix.sync()
    tx, tf = t_x.cpu().numpy(), t_f.cpu().numpy()
    return {"knn_recall": _recall(ix, qd, k, m, sample),
            "class_agreement": float((c_x.cpu().numpy() == c_f.cpu().numpy()).mean()),
            "score_rel_error": float(np.abs(tf - tx).sum() / max(1, np.abs(tx).sum())),
            "score_max_abs_error": int(np.abs(tf - tx).max())}


def part_fp8(ref, labels, shortlists, k, q_imgs, reps, sample, rows):
    import torch
    w = synth.workload("caltech256-like").with_query_imgs(q_imgs)
    q, off, _ = synth.query_set(w)
    qd, od = torch.from_numpy(q).cuda(), torch.from_numpy(off).cuda()
    with lnbnn.Index(torch.from_numpy(ref).cuda(), torch.from_numpy(labels).cuda(), w.n_classes) as ix:
        ix.prepare_fp8()
        t = _timed(lambda: ix.lnbnn_classify(qd, od, k), reps)
        _emit(rows, {"part": "fp8", "form": "exact", "k": k, "queries": len(q), "seconds": t,
                     "desc_per_s": len(q) / t})
        for m in shortlists:
            t = _timed(lambda: ix.lnbnn_classify(qd, od, k, shortlist=m), reps)
            rec = {"part": "fp8", "form": "fp8", "shortlist": m, "k": k, "queries": len(q), "seconds": t,
                   "desc_per_s": len(q) / t, "recall_sample": sample}
            rec.update(_accuracy(ix, qd, od, k, m, sample))
            _emit(rows, rec)


def part_logodds(ref, labels, betas, q_imgs, reps, rows):
    import torch
    w = synth.workload("caltech256-like").with_query_imgs(q_imgs)
    q, off, _ = synth.query_set(w)
    qd, od = torch.from_numpy(q).cuda(), torch.from_numpy(off).cuda()
    C = w.n_classes
    with lnbnn.Index(torch.from_numpy(ref).cuda(), torch.from_numpy(labels).cuda(), C) as ix:
        _, c_nbnn = ix.nbnn_classify(qd, od)
        c_nbnn = c_nbnn.cpu().numpy()
        for beta in betas:
            for pos in (False, True):
                t = _timed(lambda: ix.nbnn_logodds_classify(qd, od, beta, pos), reps)
                ix.profile_enable(True)
                _, c, n = ix.nbnn_logodds_classify(qd, od, beta, pos)
                prof = ix.profile_read()
                ix.profile_enable(False)
                ix.sync()
                _emit(rows, {"part": "logodds", "beta": beta, "positive_only": pos, "queries": len(q),
                             "seconds": t, "desc_per_s": len(q) / t,
                             "other_share": prof["other_ms"] / max(1e-9, prof["other_ms"] + prof["search_ms"]),
                             "increments_per_desc": float(n.cpu().numpy().sum()) / len(q), "classes": C,
                             "agreement_with_nbnn": float((c.cpu().numpy() == c_nbnn).mean())})


def part_single(ref, labels, sizes, ks, reps, rows):
    import torch
    w = synth.workload("caltech256-like")
    with lnbnn.Index(torch.from_numpy(ref).cuda(), torch.from_numpy(labels).cuda(), w.n_classes) as ix:
        ix.prepare_fp8()
        for n in sizes:
            qd = torch.from_numpy(synth.query_image(w, 7, n)).cuda()
            for k in ks:
                m = {10: 32, 50: 64, 100: 128}.get(k, 2 * (k + 1))
                for form, sl in (("exact", None), ("fp8", m)):
                    t = _timed(lambda: ix.knn_search(qd, k + 1, shortlist=sl), reps)
                    ix.sync()
                    _emit(rows, {"part": "single", "descriptors": n, "k": k, "form": form, "shortlist": sl,
                                 "splits": ix.plan_splits(n), "ms": t * 1e3})


def part_uneven(ref, labels, k, m, reps, sample, rows):
    import torch
    w = synth.workload("batched-uneven")
    q, off, _ = synth.query_set(w)
    qd, od = torch.from_numpy(q).cuda(), torch.from_numpy(off).cuda()
    with lnbnn.Index(torch.from_numpy(ref).cuda(), torch.from_numpy(labels).cuda(), w.n_classes) as ix:
        ix.prepare_fp8()
        for tuned in (False, True):
            tune = ix.autotune() if tuned else None
            for form, sl in (("exact", None), ("fp8", m)):
                t = _timed(lambda: ix.lnbnn_classify(qd, od, k, shortlist=sl), reps)
                rec = {"part": "uneven", "form": form, "shortlist": sl, "autotuned": tuned, "images": len(off) - 1,
                       "queries": len(q), "splits": ix.plan_splits(len(q)), "seconds": t,
                       "desc_per_s": len(q) / t, "images_per_s": (len(off) - 1) / t}
                if tune:
                    rec["tuning"] = tune
                if form == "fp8" and not tuned:
                    rec.update(_accuracy(ix, qd, od, k, m, sample))
                _emit(rows, rec)


def tables(rows) -> str:
    out = []
    kc = [r for r in rows if r["part"] == "kc"]
    if kc:
        out.append("| C | N | k | Local NBNN desc/s | TFLOP/s |\n|---|---|---|---|---|")
        for r in kc:
            k = r["k"] if r["method"] == "local" else "NBNN"
            out.append(f"| {r['C']} | {r['n_ref']:,} | {k} | {r['desc_per_s']:,.0f} | {r['tflops']:.0f} |")
    fp = [r for r in rows if r["part"] == "fp8"]
    if fp:
        out.append("\n| form | m | desc/s | recall (k+1) | class agreement | score rel. error |\n|---|---|---|---|---|---|")
        for r in fp:
            out.append(f"| {r['form']} | {r.get('shortlist', '')} | {r['desc_per_s']:,.0f} | {r.get('knn_recall', '')} "
                       f"| {r.get('class_agreement', '')} | {r.get('score_rel_error', '')} |")
    lo = [r for r in rows if r["part"] == "logodds"]
    if lo:
        out.append("\n| beta | increments | desc/s | share outside the scan | increments per descriptor "
                   "| class agreement with NBNN |\n|---|---|---|---|---|---|")
        for r in lo:
            out.append(f"| {r['beta']:g} | {'positive' if r['positive_only'] else 'all'} | {r['desc_per_s']:,.0f} "
                       f"| {r['other_share']:.3f} | {r['increments_per_desc']:.1f} of {r['classes']} "
                       f"| {r['agreement_with_nbnn']:.3f} |")
    si = [r for r in rows if r["part"] == "single"]
    if si:
        out.append("\n| descriptors | splits | k | exact ms | FP8 ms (m) |\n|---|---|---|---|---|")
        for r in si:
            if r["form"] == "exact":
                f = next((x for x in si if x["form"] == "fp8" and x["descriptors"] == r["descriptors"]
                          and x["k"] == r["k"]), None)
                out.append(f"| {r['descriptors']:,} | {r['splits']} | {r['k']} | {r['ms']:.2f} "
                           f"| {f['ms']:.2f} ({f['shortlist']}) |" if f else "")
    un = [r for r in rows if r["part"] == "uneven"]
    if un:
        out.append("\n| form | autotuned | splits | desc/s | images/s |\n|---|---|---|---|---|")
        for r in un:
            out.append(f"| {r['form']} | {r['autotuned']} | {r['splits']} | {r['desc_per_s']:,.0f} "
                       f"| {r['images_per_s']:.1f} |")
    return "\n".join(out)


def main():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--parts", default="kc,fp8,logodds,single,uneven")
    p.add_argument("--classes", default="32,64,128,256")
    p.add_argument("--ks", default="1,2,5,10,20,50,100")
    p.add_argument("--shortlists", default="16,32,64,128")
    p.add_argument("--betas", default="1e-6,1e-5,1e-4,1e-3")
    p.add_argument("--query-images", type=int, default=100)
    p.add_argument("--reps", type=int, default=3)
    p.add_argument("--k", type=int, default=10)
    p.add_argument("--recall-sample", type=int, default=8192)
    a = p.parse_args()
    lnbnn.load_library()
    parts = a.parts.split(",")
    ref, labels = synth.reference_set(synth.workload("caltech256-like"))
    rows: list = []
    if "kc" in parts:
        part_kc(ref, labels, [int(c) for c in a.classes.split(",")], [int(k) for k in a.ks.split(",")],
                a.query_images, a.reps, rows)
    if "fp8" in parts:
        part_fp8(ref, labels, [int(m) for m in a.shortlists.split(",")], a.k, a.query_images, a.reps,
                 a.recall_sample, rows)
    if "logodds" in parts:
        part_logodds(ref, labels, [float(b) for b in a.betas.split(",")], a.query_images, a.reps, rows)
    if "single" in parts:
        part_single(ref, labels, [100, 632, 1000, 4000], [10, 50, 100], a.reps, rows)
    if "uneven" in parts:
        part_uneven(ref, labels, a.k, 32, a.reps, a.recall_sample, rows)
    print(tables(rows), flush=True)


if __name__ == "__main__":
    main()
