"""Continuous-batching server for Local NBNN (Alg. 2) / NBNN (Alg. 1) queries.

The merged index stays resident in HBM.  The server owns a few *slots*; each
slot is a workspace (device scratch that a call uses without allocating), a
CUDA stream, device buffers and pinned host buffers for one batch of at most
``max_batch_queries`` descriptors.  Its request loop admits arriving images in
arrival order into the batch of the next free slot while the slot has room
(admission by free workspace memory), and launches the batch as one
host->device copy, one classify call and one device->host copy on the slot's
stream.  Batches on different slots overlap on the GPU, and requests that
arrive while batches are in flight are admitted as soon as a slot frees up.

With ``graphs=True`` each slot captures, per query-count bucket (multiples
of 128 descriptors: every one up to 4,096, then about 25% apart), one CUDA
graph holding the copies and the classify call; a batch is padded up to its bucket with zero descriptors
that form one extra image, whose scores are dropped.  The padding changes no real image's result: Alg. 2 scores every
descriptor on its own, and a descriptor counts only toward its own image.

All classification runs in the CUDA library; this module moves bytes and
keeps time.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    """One query image: its descriptors and the time it arrived (seconds)."""

    rid: int
    descriptors: np.ndarray  # uint8 [n, row bytes of the index: 128, or 130 with a location]
    arrival: float
    totals: np.ndarray | None = None
    cls: int | None = None
    done: float | None = None
    batch: int | None = None  # id of the batch that served it


def take_batch(pending: collections.deque, max_queries: int, max_images: int) -> list:
    """Admit requests from the front of ``pending`` (arrival order) while the
    batch stays within ``max_queries`` descriptors and ``max_images`` images.
    A request that alone exceeds ``max_queries`` can never be served: raise."""
    batch, n = [], 0
    while pending and len(batch) < max_images:
        m = len(pending[0].descriptors)
        if m > max_queries:
            raise ValueError(f"request {pending[0].rid} has {m} descriptors, more than a batch holds ({max_queries})")
        if n + m > max_queries:
            break
        batch.append(pending.popleft())
        n += m
    return batch


def graph_buckets(max_queries: int, granule: int = 128, ratio: float = 1.25, fine_upto: int = 4096) -> list[int]:
    """Query counts the server captures graphs for: every multiple of
    ``granule`` up to ``fine_upto`` (a lone image pads to its next query tile
    only), then multiples of ``granule`` growing by about ``ratio`` (padding a
    batch to its bucket wastes at most that fraction of the search), ending at
    ``max_queries``."""
    out, b = [], granule
    while b < max_queries:
        out.append(b)
        b = b + granule if b < fine_upto else max(b + granule, -(-int(b * ratio) // granule) * granule)
    out.append(max_queries)
    return out


def bucket_of(n: int, buckets: list[int]) -> int:
    """Smallest bucket that holds n descriptors."""
    for b in buckets:
        if n <= b:
            return b
    raise ValueError(f"{n} descriptors exceed the largest bucket {buckets[-1]}")


@dataclass
class _Slot:
    ws: object
    stream: object
    q_host: object
    off_host: object
    tot_host: object
    cls_host: object
    q_dev: object
    off_dev: object
    tot_dev: object
    cls_dev: object
    event: object
    graphs: dict = field(default_factory=dict)
    batch: list = field(default_factory=list)
    launched: float = 0.0


class Server:
    """Continuous-batching classifier over one ``lnbnn.Index``.

    method: "local" (Alg. 2 with neighbourhood k) or "nbnn" (Alg. 1).
    shortlist: None for the exact search, else the FP8 shortlist length of
    the approximate search ("local" only; the index needs prepare_fp8()).
    slots: batches that can be in flight at once.
    max_batch_queries / max_batch_images: the capacity of one slot.
    graphs: replay captured CUDA graphs (one per slot and query-count
    bucket, see ``graph_buckets``) instead of launching each call.
    """

    def __init__(self, index, k: int = 10, method: str = "local", slots: int = 2, max_batch_queries: int = 16384,
                 max_batch_images: int = 256, graphs: bool = False, shortlist: int | None = None):
        import torch

        if method not in ("local", "nbnn"):
            raise ValueError("method must be 'local' or 'nbnn'")
        if shortlist is not None and method != "local":
            raise ValueError("the FP8 shortlist search serves Local NBNN only")
        self.shortlist = shortlist
        self.index, self.k, self.method = index, int(k), method
        self.max_q, self.max_img = int(max_batch_queries), int(max_batch_images)
        self.use_graphs = bool(graphs)
        self.buckets = graph_buckets(self.max_q)
        C = index.n_classes
        D = getattr(index, "row_bytes", 128)  # 130 for a location-weighted index
        dev = torch.device("cuda", torch.cuda.current_device())
        # Graph mode adds one image that holds the padding descriptors.
        n_img_cap = self.max_img + 1
        self.slots = []
        for _ in range(slots):
            self.slots.append(_Slot(
                ws=index.workspace(self.max_q, max(self.k, (shortlist or 0) - 1)),
                stream=torch.cuda.Stream(dev),
                q_host=torch.zeros((self.max_q, D), dtype=torch.uint8).pin_memory(),
                off_host=torch.empty((n_img_cap + 1,), dtype=torch.int64).pin_memory(),
                tot_host=torch.empty((n_img_cap, C), dtype=torch.int64).pin_memory(),
                cls_host=torch.empty((n_img_cap,), dtype=torch.int32).pin_memory(),
                q_dev=torch.empty((self.max_q, D), dtype=torch.uint8, device=dev),
                off_dev=torch.empty((n_img_cap + 1,), dtype=torch.int64, device=dev),
                tot_dev=torch.empty((n_img_cap, C), dtype=torch.int64, device=dev),
                cls_dev=torch.empty((n_img_cap,), dtype=torch.int32, device=dev),
                event=torch.cuda.Event()))
        self.pending: collections.deque[Request] = collections.deque()
        self.batches = 0
        # One record per batch: (launch time, completion time, images, descriptors).
        self.log: list[tuple[float, float, int, int]] = []
        if self.use_graphs:
            self._capture_all()

    def close(self) -> None:
        for s in self.slots:
            s.graphs.clear()
            s.ws.close()
        self.slots = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------ one batch

    def _enqueue(self, slot: _Slot, n: int, b: int) -> None:
        """Copies + classify + copies of a batch of n descriptors in b images,
        on the current stream (the slot's)."""
        s = slot.stream
        slot.q_dev[:n].copy_(slot.q_host[:n], non_blocking=True)
        slot.off_dev[:b + 1].copy_(slot.off_host[:b + 1], non_blocking=True)
        out = (slot.tot_dev[:b], slot.cls_dev[:b])
        if self.method == "local":
            self.index.lnbnn_classify(slot.q_dev[:n], slot.off_dev[:b + 1], self.k, stream=s, out=out,
                                      workspace=slot.ws, shortlist=self.shortlist)
        else:
            self.index.nbnn_classify(slot.q_dev[:n], slot.off_dev[:b + 1], stream=s, out=out, workspace=slot.ws)
        slot.tot_host[:b].copy_(slot.tot_dev[:b], non_blocking=True)
        slot.cls_host[:b].copy_(slot.cls_dev[:b], non_blocking=True)

    def _capture_all(self) -> None:
        """Capture, per slot and bucket, the batch of ``max_img`` + 1 images
        over the bucket's descriptor count.  Unused images are empty."""
        import torch

        b = self.max_img + 1
        for slot in self.slots:
            slot.off_host.zero_()
            slot.off_host[b] = self.buckets[0]  # all descriptors in the last image
            with torch.cuda.stream(slot.stream):  # one eager run: lazy initialisation happens outside capture
                self._enqueue(slot, self.buckets[0], b)
            slot.stream.synchronize()
            for n in self.buckets:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=slot.stream):
                    self._enqueue(slot, n, b)
                slot.graphs[n] = g
        torch.cuda.synchronize()
        self.index.sync()

    def _launch(self, slot: _Slot, now: float) -> None:
        """Fill the slot's batch from the pending queue and launch it."""
        import torch

        batch = take_batch(self.pending, self.max_q, self.max_img)
        if not batch:
            return
        qh, oh = slot.q_host.numpy(), slot.off_host.numpy()
        oh[0] = 0
        for i, r in enumerate(batch):
            m = len(r.descriptors)
            qh[oh[i]:oh[i] + m] = r.descriptors
            oh[i + 1] = oh[i] + m
        b, n = len(batch), int(oh[len(batch)])
        with torch.cuda.stream(slot.stream):
            if self.use_graphs:
                nb = bucket_of(n, self.buckets)
                qh[n:nb] = 0  # padding descriptors: the extra image b
                oh[b + 1:] = nb
                slot.graphs[nb].replay()
            else:
                self._enqueue(slot, n, b)
            slot.event.record(slot.stream)
        for r in batch:
            r.batch = self.batches
        slot.batch, slot.launched = batch, now
        self.batches += 1

    def _complete(self, slot: _Slot, now: float) -> list[Request]:
        b = len(slot.batch)
        tot, cls = slot.tot_host.numpy()[:b], slot.cls_host.numpy()[:b]
        for i, r in enumerate(slot.batch):
            r.totals, r.cls, r.done = tot[i].copy(), int(cls[i]), now
        self.log.append((slot.launched, now, b, sum(len(r.descriptors) for r in slot.batch)))
        done, slot.batch = slot.batch, []
        return done

    # ------------------------------------------------------------ request loop

    def run(self, requests: list[Request], clock=time.perf_counter) -> list[Request]:
        """Serve ``requests``, each admitted once its arrival time (seconds
        after the start of the call) has passed.  Returns them completed."""
        order = sorted(requests, key=lambda r: r.arrival)
        t0 = clock()
        nxt, finished = 0, []
        while len(finished) < len(order):
            now = clock() - t0
            while nxt < len(order) and order[nxt].arrival <= now:
                self.pending.append(order[nxt])
                nxt += 1
            progressed = False
            for slot in self.slots:
                if slot.batch and slot.event.query():
                    finished += self._complete(slot, clock() - t0)
                    progressed = True
                if not slot.batch and self.pending:
                    self._launch(slot, clock() - t0)
                    progressed = True
            if not progressed and not any(slot.batch for slot in self.slots):
                time.sleep(50e-6)  # nothing on the GPU: wait for arrivals; with a batch in flight, poll
        self.index.sync()
        return finished


def poisson_requests(w, rate: float, n: int, seed: int = 0, first_image: int = 0) -> list[Request]:
    """n query images of workload w (its descriptor-count rule) arriving as a
    Poisson process of ``rate`` images per second, the first at time 0."""
    from . import synth

    rng = np.random.default_rng([seed, 7, int(rate * 1000)])
    gaps = rng.exponential(1.0 / rate, size=n)
    arrivals = np.concatenate([[0.0], np.cumsum(gaps[1:])])
    counts = synth.query_counts(w.with_query_imgs(first_image + n))[first_image:]
    return [Request(i, synth.query_image(w, first_image + i, int(counts[i])), float(arrivals[i])) for i in range(n)]


def max_in_flight(log) -> int:
    """Most batches on the GPU at one time, from ``Server.log``."""
    ev = sorted([(t0, 1) for t0, _, _, _ in log] + [(t1, -1) for _, t1, _, _ in log], key=lambda e: (e[0], e[1]))
    cur = best = 0
    for _, d in ev:
        cur += d
        best = max(best, cur)
    return best


def latency_stats(done: list[Request], log=None) -> dict:
    """p50 / p99 latency (arrival to result on the host) and throughput."""
    lat = np.array([r.done - r.arrival for r in done])
    span = max(r.done for r in done) - min(r.arrival for r in done)
    out = {"images": len(done), "images_per_s": len(done) / span,
           "query_descriptors_per_s": sum(len(r.descriptors) for r in done) / span,
           "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3)}
    if log:
        out["batches"] = len(log)
        out["mean_images_per_batch"] = float(np.mean([b for _, _, b, _ in log]))
        out["max_batches_in_flight"] = max_in_flight(log)
    return out
