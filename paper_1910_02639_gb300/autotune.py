"""Autotuner for the batched b-tree: per size class of particle set, the
bucket size s, the empty-cell limit beta (Eq. 4), the find work-unit size
(queries searched together), whether sibling leaves share work units, and
the find block shape (8 warps and a 1024-candidate window, or 4 warps and
512) that minimise build + find + density time.

None of the knobs changes a result: the neighbour lists are defined without
reference to the tree, and the density of a particle is summed in the order
of its sorted list.  So the tuner only times.

Search: coordinate descent from (wide shape, no packing, s = 16, beta = 0.5,
32 queries) -- the block shape first, then packing, s, beta and the
work-unit size -- on a sample of the sets of each class (half-decades of n x
three classes of the spread of h within the set), each candidate timed with
CUDA events after a
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
    "pack_leaves": (False, True),
}
START = {"bucket_size": 16, "beta": 0.5, "group_size": 32, "find_compact": False,
         "pack_leaves": False}


def size_class(n: int) -> int:
    """Half-decade of n: 6 for [1e3, 3.16e3), 7 for [3.16e3, 1e4), ..."""
    return int(math.floor(2.0 * math.log10(max(int(n), 1))))


def spread_class(h) -> int:
    """How much h varies within a set (std / mean): 0 below 0.05 (uniform
    resolution), 1 below 0.5, 2 above (strongly adaptive: cores and wide
    outskirts).  A set's best parameters depend on this as much as on n."""
    import numpy as np
    h = np.asarray(h, dtype=np.float64)
    if h.size == 0:
        return 0
    mu = float(h.mean())
    cv = float(h.std()) / mu if mu > 0 else 0.0
    return 0 if cv < 0.05 else (1 if cv < 0.5 else 2)


def set_class(s) -> tuple:
    """Tuning class of a particle set: (size class, spread class)."""
    return (size_class(s.n), spread_class(s.h))


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
            for key in ("find_compact", "pack_leaves", "bucket_size", "beta", "group_size"):
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
                by.setdefault(set_class(s), []).append(s)
        for c in sorted(by):
            self.table[c] = self.tune_class(by[c])
        return self.table

    def params_for(self, sets) -> list:
        out = []
        for s in sets:
            p = dict(DEFAULT_PARAMS)
            e = self.table.get(set_class(s)) if s.n > 0 else None
            if e:
                p.update(bucket_size=e["bucket_size"], beta=e["beta"], group_size=e["group_size"],
                         find_compact=e["find_compact"], pack_leaves=e.get("pack_leaves", False))
            out.append(p)
        return out

    # ------------------------------------------------------------ storage
    def save(self, path: str):
        with open(path, "w") as f:
            json.dump({"%d,%d" % k: v for k, v in self.table.items()}, f, indent=1, sort_keys=True)

    def load(self, path: str):
        with open(path) as f:
            self.table = {tuple(int(v) for v in k.split(",")): e for k, e in json.load(f).items()}
        return self.table
