"""Autotuner for the batched b-tree: per size class of particle set, the
bucket size s, the empty-cell limit beta (Eq. 4), the find work-unit size
(queries searched together) and the find block shape (8 warps and a
1024-candidate window, or 4 warps and 512) that minimise build + find +
density time.

None of the knobs changes a result: the neighbour lists are defined without
reference to the tree, and the density of a particle is summed in the order
of its sorted list.  So the tuner only times.

Search: coordinate descent from (wide shape, s = 16, beta = 0.5, 32 queries)
-- the block shape first, then s, beta and the work-unit size -- on a sample
of the sets of each size
class (half-decades of n), each candidate timed with CUDA events after a
warm-up run; a change is kept only if it is more than `margin` (3 %) faster
than the best so far, so that timing noise does not move the choice.  The
table maps a size class to its parameters and can be saved and loaded as
JSON.
"""
from __future__ import annotations

import json
import math

from .batch import DEFAULT_PARAMS, DeviceSets

SPACE = {
    "bucket_size": (8, 16, 32, 64),
    "beta": (0.25, 0.5, 0.75),
    "group_size": (16, 32),
    "find_compact": (False, True),
}
START = {"bucket_size": 16, "beta": 0.5, "group_size": 32, "find_compact": False}


def size_class(n: int) -> int:
    """Half-decade of n: 6 for [1e3, 3.16e3), 7 for [3.16e3, 1e4), ..."""
    return int(math.floor(2.0 * math.log10(max(int(n), 1))))


class Tuner:
    def __init__(self, device, ngmax: int, stream=None, reps: int = 3,
                 sample_particles: int = 2_000_000, space=None, margin: float = 0.03):
        self.device = device
        self.ngmax = ngmax
        self.stream = stream
        self.reps = reps
        self.sample_particles = sample_particles
        self.space = dict(space or SPACE)
        self.margin = margin
        self.table: dict[int, dict] = {}
        self.trials = 0

    # ------------------------------------------------------------ timing
    def _time(self, ds: DeviceSets, params: dict) -> float:
        import torch
        st = self.stream or torch.cuda.current_stream(ds.device)
        ds.run_batched(params, stream=st)  # warm-up (and buffer growth)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(self.reps):
            ds.run_batched(params, stream=st)
        e1.record(st)
        e1.synchronize()
        self.trials += 1
        return e0.elapsed_time(e1) / self.reps

    def _sample(self, sets):
        """Sets of one class, largest share first, up to the particle budget."""
        out, tot = [], 0
        for s in sorted(sets, key=lambda s: -s.n):
            if out and tot + s.n > self.sample_particles:
                continue
            out.append(s)
            tot += s.n
        return out

    # ------------------------------------------------------------ search
    def tune_class(self, sets) -> dict:
        ds = DeviceSets(self._sample(sets), self.device, self.ngmax)
        try:
            cur = dict(START)
            best = self._time(ds, dict(DEFAULT_PARAMS, **cur))
            for key in ("find_compact", "bucket_size", "beta", "group_size"):
                for v in self.space[key]:
                    if v == cur[key]:
                        continue
                    cand = dict(cur, **{key: v})
                    t = self._time(ds, dict(DEFAULT_PARAMS, **cand))
                    if t < best * (1.0 - self.margin):  # a change must beat timing noise
                        best, cur = t, cand
            return dict(cur, ms=best)
        finally:
            ds.free()

    def tune(self, sets) -> dict:
        by = {}
        for s in sets:
            if s.n > 0:
                by.setdefault(size_class(s.n), []).append(s)
        for c in sorted(by):
            self.table[c] = self.tune_class(by[c])
        return self.table

    def params_for(self, sets) -> list:
        out = []
        for s in sets:
            p = dict(DEFAULT_PARAMS)
            e = self.table.get(size_class(s.n))
            if e:
                p.update(bucket_size=e["bucket_size"], beta=e["beta"], group_size=e["group_size"],
                         find_compact=e["find_compact"])
            out.append(p)
        return out

    # ------------------------------------------------------------ storage
    def save(self, path: str):
        with open(path, "w") as f:
            json.dump({str(k): v for k, v in self.table.items()}, f, indent=1, sort_keys=True)

    def load(self, path: str):
        with open(path) as f:
            self.table = {int(k): v for k, v in json.load(f).items()}
        return self.table
