"""Serving: a continuous-batching request loop for build + find + density jobs.

Requests (one particle set each) wait in a FIFO queue.  Whenever one of the
`slots` workers is idle, the scheduler admits the longest prefix of the
waiting requests that fits both the free-HBM budget and the per-batch particle
limit, and hands that batch to the worker.  The worker copies the inputs from
pinned host memory on its own CUDA stream, builds all of the batch's sets in
one ``btree_build_batched`` call, runs one fused find + density over them and
waits for its stream.  Requests that arrive while batches are on the GPU are
admitted as slots and memory free up, and batches on different slots overlap
on the device.

Results stay in device memory (views of the batch's output buffers) until the
client releases them; the batch's inputs and outputs return to the budget
when all of its results are released.  Each slot keeps its tree between
batches; the tree's bound (tree_bytes) stays charged to the slot, and a batch
is charged only for the growth of its slot's tree.  Every batch's span on the
device (CUDA events on its slot's stream) is kept in Server.timeline.  A request the library rejects (non-finite
coordinates or smoothing lengths) fails alone: its batch is re-run request by
request and only it returns an error result.  Each request's lists, counts
and densities are bit-identical to those of the same set run alone: sets in a
batch do not interact, and every per-particle result depends only on its own
set.
"""
from __future__ import annotations

import math
import queue
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import BtreeError, btree_build, btree_build_batched, btree_find_neighbors_density


def io_bytes(n: int, ngmax: int) -> int:
    """Device bytes of one request's inputs (x, y, z, h, m) and outputs (rows,
    counts, densities): held until its result is released."""
    return int(n) * (5 * 4 + 4 * ngmax + 4 + 4) + (1 << 20)


def tree_bytes(n: int) -> int:
    """A generous bound on a tree's buffers for n particles (sorted copy,
    permutation, working buffers, nodes, sub-cells, work units).  A slot keeps
    its tree between batches, so this stays charged to the slot."""
    return int(n) * 96 + (1 << 20)


def request_bytes(n: int, ngmax: int) -> int:
    """Device bytes one request needs on a slot that holds no tree yet."""
    return io_bytes(n, ngmax) + tree_bytes(n)


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the replay
    x: object                      # pinned host float32 tensors
    y: object
    z: object
    h: object
    m: object
    params: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.numel())


@dataclass
class Result:
    rid: int
    n: int
    nb: object                     # device int32 [n * ngmax] (view)
    cnt: object                    # device int32 [n]
    rho: object                    # device float32 [n]
    arrival: float
    admitted: float
    done: float
    batch: int
    batch_size: int
    _batch_ref: object = None
    error: str | None = None       # set when the request failed (then nb/cnt/rho are None)
    slot: int = -1                 # the worker slot that ran it

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def make_request(rid, arrival, s, params=None):
    """Pinned host copies of a ParticleSet."""
    import torch
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()
    return Request(rid, float(arrival), pin(s.x), pin(s.y), pin(s.z), pin(s.h), pin(s.m),
                   dict(params or {}))


class _Batch:
    """Device buffers of one admitted batch; freed when all results go."""

    def __init__(self, server, reqs, nbytes):
        self.server = server
        self.reqs = reqs
        self.nbytes = nbytes
        self.live = len(reqs)
        self.lock = threading.Lock()

    def release_one(self):
        with self.lock:
            self.live -= 1
            last = self.live == 0
        if last:
            self.bufs = None
            self.server._return_bytes(self.nbytes)


class Server:
    def __init__(self, device="cuda:0", ngmax: int = 256, slots: int = 4,
                 hbm_budget: int | None = None, max_batch_particles: int = 8_000_000,
                 reserve_bytes: int = 4 << 30, params_for=None):
        import torch
        self.device = torch.device(device)
        self.ngmax = int(ngmax)
        self.slots = int(slots)
        self.max_batch_particles = int(max_batch_particles)
        free, _ = torch.cuda.mem_get_info(self.device)
        budget = free - reserve_bytes
        self.budget = int(min(budget, hbm_budget) if hbm_budget else budget)
        if self.budget <= 0:
            raise RuntimeError("no HBM left for the serving budget")
        self.params_for = params_for  # optional: n -> per-set parameter dict
        self._free_bytes = self.budget
        self._cv = threading.Condition()
        self._waiting: list[Request] = []
        self._done: "queue.Queue[Result]" = queue.Queue()
        self._idle = list(range(self.slots))
        self._work = [queue.Queue() for _ in range(self.slots)]
        self._streams = [torch.cuda.Stream(self.device) for _ in range(self.slots)]
        self._trees = [None] * self.slots
        self._slot_tree = [0] * self.slots  # bytes charged for each slot's kept tree
        # per batch on the device: (batch, slot, start_ms, end_ms, requests),
        # from CUDA events on the slot's stream, relative to start_clock()
        self.timeline: list[tuple] = []
        self._ref = None
        self._t0 = None
        self._nbatch = 0
        self._stop = False
        self._threads = [threading.Thread(target=self._worker, args=(k,), daemon=True)
                         for k in range(self.slots)]
        self.errors: list[BaseException] = []
        for t in self._threads:
            t.start()

    # ------------------------------------------------------------ clock
    def start_clock(self, t0: float | None = None):
        import torch
        self._t0 = time.perf_counter() if t0 is None else t0
        self._ref = torch.cuda.Event(enable_timing=True)
        self._ref.record(torch.cuda.current_stream(self.device))

    def now(self) -> float:
        return time.perf_counter() - self._t0

    # ------------------------------------------------------------ client side
    def submit(self, req: Request):
        if request_bytes(req.n, self.ngmax) > self.budget:
            raise ValueError(f"request {req.rid} ({req.n} particles) exceeds the HBM budget")
        with self._cv:
            self._waiting.append(req)
            self._admit_locked()

    def poll(self, timeout: float | None = None):
        """Next finished Result (blocking up to `timeout`), or None."""
        try:
            return self._done.get(timeout=timeout)
        except queue.Empty:
            return None

    def release(self, res: Result):
        """Give a result's device memory back (after the client is done);
        failed requests hold none."""
        b = res._batch_ref
        res._batch_ref = None
        res.nb = res.cnt = res.rho = None
        if b is not None:
            b.release_one()

    def close(self):
        self._stop = True
        for q in self._work:
            q.put(None)
        for t in self._threads:
            t.join(timeout=30)
        for tr in self._trees:
            if tr is not None:
                tr.free()

    # ------------------------------------------------------------ scheduler
    def _return_bytes(self, nbytes):
        with self._cv:
            self._free_bytes += nbytes
            self._admit_locked()

    def _admit_locked(self):
        """FIFO admission: while a slot is idle, take the longest prefix of the
        waiting queue that fits the free budget and the batch limit.  A batch
        costs its inputs and outputs plus whatever its tree needs beyond the
        tree the slot already holds (that stays charged to the slot)."""
        while self._idle and self._waiting:
            slot = self._idle[0]
            have = self._slot_tree[slot]
            take, nbytes, npart, grow = [], 0, 0, 0
            for r in self._waiting:
                b = io_bytes(r.n, self.ngmax)
                g = max(0, tree_bytes(npart + r.n) - have)
                if nbytes + b + g > self._free_bytes:
                    break
                if take and npart + r.n > self.max_batch_particles:
                    break
                take.append(r)
                nbytes += b
                npart += r.n
                grow = g
            if not take:
                # the head waits for memory -- unless trees kept by other idle
                # slots hold it: free those and try again
                if self._reclaim_locked(keep=slot):
                    continue
                return
            del self._waiting[:len(take)]
            self._free_bytes -= nbytes + grow
            self._slot_tree[slot] += grow
            self._idle.pop(0)
            self._nbatch += 1
            t_adm = self.now() if self._t0 is not None else 0.0
            self._work[slot].put((self._nbatch, take, nbytes, t_adm))

    def _reclaim_locked(self, keep: int) -> bool:
        """Free the trees of idle slots other than `keep` (no work of theirs
        is in flight); True when that returned any bytes."""
        got = 0
        for k in self._idle:
            if k != keep and self._slot_tree[k] > 0:
                if self._trees[k] is not None:
                    self._trees[k].free()
                    self._trees[k] = None
                got += self._slot_tree[k]
                self._slot_tree[k] = 0
        self._free_bytes += got
        return got > 0

    # ------------------------------------------------------------ workers
    def _worker(self, slot):
        import torch
        torch.cuda.set_device(self.device)
        st = self._streams[slot]
        while True:
            job = self._work[slot].get()
            if job is None:
                return
            bid, reqs, nbytes, t_adm = job
            try:
                self._run_batch(slot, st, bid, reqs, nbytes, t_adm)
            except BtreeError:
                # a request of the batch failed (e.g. non-finite input): run
                # each request alone, within the memory the batch holds, so
                # that only the bad ones fail
                held = nbytes
                for r in reqs:
                    one = io_bytes(r.n, self.ngmax)
                    try:
                        self._run_batch(slot, st, bid, [r], one, t_adm)
                        held -= one  # now owned by that result's buffers
                    except BtreeError as e1:
                        self._done.put(Result(r.rid, r.n, None, None, None, r.arrival, t_adm,
                                              self.now(), bid, 1, None, error=str(e1)))
                    except BaseException as e1:  # not a request error: report it
                        self.errors.append(e1)
                self._return_bytes(held)
            except BaseException as e:  # reported to the caller, slot stays usable
                self.errors.append(e)
                self._return_bytes(nbytes)
            with self._cv:
                self._idle.append(slot)
                self._admit_locked()

    def _run_batch(self, slot, st, bid, reqs, nbytes, t_adm):
        import torch
        g = self.ngmax
        sizes = [r.n for r in reqs]
        off = np.zeros(len(reqs) + 1, np.int64)
        off[1:] = np.cumsum(sizes)
        n = int(off[-1])
        n1 = max(n, 1)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            ev0.record(st)
            dev = self.device
            x, y, z, h, m = (torch.empty(n1, dtype=torch.float32, device=dev) for _ in range(5))
            for r, a, b in zip(reqs, off[:-1], off[1:]):
                a, b = int(a), int(b)
                for d, s in ((x, r.x), (y, r.y), (z, r.z), (h, r.h), (m, r.m)):
                    d[a:b].copy_(s, non_blocking=True)
            nb = torch.empty(n1 * g, dtype=torch.int32, device=dev)
            cnt = torch.empty(n1, dtype=torch.int32, device=dev)
            rho = torch.empty(n1, dtype=torch.float32, device=dev)
            params = [dict(r.params) if r.params else
                      (self.params_for(r.n) if self.params_for else {}) for r in reqs]
            self._trees[slot] = btree_build_batched(x[:n], y[:n], z[:n], h[:n], off, params,
                                                    stream=st, tree=self._trees[slot])
            btree_find_neighbors_density(self._trees[slot], m[:n], g, nb, cnt, rho, stream=st)
            ev1.record(st)
        st.synchronize()
        t_done = self.now()
        if self._ref is not None:
            self.timeline.append((bid, slot, self._ref.elapsed_time(ev0), self._ref.elapsed_time(ev1),
                                  len(reqs)))
        batch = _Batch(self, reqs, nbytes)
        batch.bufs = (x, y, z, h, m, nb, cnt, rho)
        for r, a, b in zip(reqs, off[:-1], off[1:]):
            a, b = int(a), int(b)
            self._done.put(Result(r.rid, r.n, nb[a * g:b * g], cnt[a:b], rho[a:b], r.arrival,
                                  t_adm, t_done, bid, len(reqs), batch, slot=slot))


# ---------------------------------------------------------------- replay
def replay(server: Server, requests, on_result=None, timeout: float = 600.0):
    """Submit each request at its arrival time (wall clock from now) and
    collect every result.  `on_result(res)` is called for each finished
    request, before its memory is released.  Returns the results (their
    device views released)."""
    reqs = sorted(requests, key=lambda r: r.arrival)
    server.start_clock()
    out, i, t_end = [], 0, time.perf_counter() + timeout
    while len(out) < len(reqs):
        if time.perf_counter() > t_end:
            raise TimeoutError("replay did not finish")
        now = server.now()
        while i < len(reqs) and reqs[i].arrival <= now:
            server.submit(reqs[i])
            i += 1
        wait = (reqs[i].arrival - server.now()) if i < len(reqs) else 0.05
        res = server.poll(timeout=max(1e-4, min(wait, 0.05)))
        while res is not None:
            if on_result:
                on_result(res)
            server.release(res)
            out.append(res)
            res = server.poll(timeout=0)
        if server.errors:
            raise server.errors[0]
    return out


def replay_plain(requests, device="cuda:0", ngmax: int = 256, on_result=None,
                 params_for=None):
    """The plain path under the same arrivals: one job at a time, FIFO, each
    set copied in, built and searched alone (btree_build + fused find)."""
    import torch
    dev = torch.device(device)
    st = torch.cuda.Stream(dev)
    reqs = sorted(requests, key=lambda r: r.arrival)
    t0 = time.perf_counter()
    tree, out = None, []
    for r in reqs:
        now = time.perf_counter() - t0
        if r.arrival > now:
            time.sleep(r.arrival - now)
        t_adm = time.perf_counter() - t0
        n, g = r.n, ngmax
        p = dict(r.params) if r.params else (params_for(n) if params_for else {})
        with torch.cuda.stream(st):
            x, y, z, h, m = (s.to(dev, non_blocking=True) for s in (r.x, r.y, r.z, r.h, r.m))
            nb = torch.empty(max(n, 1) * g, dtype=torch.int32, device=dev)
            cnt = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
            rho = torch.empty(max(n, 1), dtype=torch.float32, device=dev)
            tree = btree_build(x, y, z, h, bucket_size=p.get("bucket_size", 16),
                               alpha=p.get("alpha", 0.5), beta=p.get("beta", 0.5), stream=st,
                               tree=tree)
            btree_find_neighbors_density(tree, m, g, nb, cnt, rho, stream=st)
        st.synchronize()
        res = Result(r.rid, n, nb, cnt, rho, r.arrival, t_adm, time.perf_counter() - t0, -1, 1)
        if on_result:
            on_result(res)
        res.nb = res.cnt = res.rho = None
        out.append(res)
    if tree is not None:
        tree.free()
    return out


def latency_stats(results, pairs: int):
    lat = np.array([r.latency for r in results], np.float64) * 1e3
    span = max(r.done for r in results) - min(r.arrival for r in results)
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
            "pairs_per_s": pairs / span if span > 0 else math.nan, "makespan_s": span,
            "requests": len(results)}
