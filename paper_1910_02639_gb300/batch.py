"""Many particle sets on one GPU.

`DeviceSets` holds several independent particle sets concatenated in device
memory, with output buffers for their neighbour lists, counts and densities.
It can run them two ways, with identical results:

* ``run_batched`` -- one ``btree_build_batched`` over all sets, then one fused
  find + density call (a few launches for the whole batch);
* ``run_graph`` -- the same two steps as one CUDA graph launch
  (``btree_build_find_batched``);
* ``run_plain`` -- the plain path: ``btree_build`` and the fused find for each
  set in turn, each set on its own tree.

Row i of the neighbour buffer is the i-th particle of the concatenation and
holds indices within that particle's own set.
"""
from __future__ import annotations

import numpy as np

from . import (btree_build, btree_build_batched, btree_build_find_batched,
               btree_find_neighbors_density)

DEFAULT_PARAMS = dict(bucket_size=16, alpha=0.5, beta=0.5, octree=False, group_size=0,
                      find_compact=False, dim=3, pack_leaves=False)


def offsets_of(sizes) -> np.ndarray:
    off = np.zeros(len(sizes) + 1, np.int64)
    off[1:] = np.cumsum(np.asarray(sizes, np.int64))
    return off


class DeviceSets:
    """Sets concatenated on `device` (float32 x, y, z, h, m) plus outputs."""

    def __init__(self, sets, device, ngmax: int, density: bool = True):
        import torch
        self.device = torch.device(device)
        self.ngmax = int(ngmax)
        self.sizes = [int(s.n) for s in sets]
        self.offsets = offsets_of(self.sizes)
        self.n = int(self.offsets[-1])
        cat = lambda k: np.ascontiguousarray(
            np.concatenate([getattr(s, k) for s in sets]) if sets else np.zeros(0), np.float32)
        self.x, self.y, self.z, self.h, self.m = (
            torch.from_numpy(cat(k)).to(self.device) for k in ("x", "y", "z", "h", "m"))
        n1 = max(self.n, 1)
        self.nb = torch.empty(n1 * self.ngmax, dtype=torch.int32, device=self.device)
        self.cnt = torch.empty(n1, dtype=torch.int32, device=self.device)
        self.rho = torch.empty(n1, dtype=torch.float32, device=self.device) if density else None
        self._tree = None
        self._trees = {}

    @property
    def nsets(self) -> int:
        return len(self.sizes)

    def params_list(self, params):
        if params is None:
            return [dict(DEFAULT_PARAMS) for _ in self.sizes]
        if isinstance(params, dict):
            return [dict(DEFAULT_PARAMS, **params) for _ in self.sizes]
        return [dict(DEFAULT_PARAMS, **p) for p in params]

    def run_batched(self, params=None, stream=None):
        """One batched build + one fused find over every set."""
        self._tree = btree_build_batched(self.x, self.y, self.z, self.h, self.offsets,
                                         self.params_list(params), stream=stream, tree=self._tree)
        btree_find_neighbors_density(self._tree, self.m, self.ngmax, self.nb, self.cnt, self.rho,
                                     stream=stream)
        return self._tree

    def run_graph(self, params=None, stream=None):
        """The batched build and the fused find as one CUDA graph launch."""
        self._tree = btree_build_find_batched(self.x, self.y, self.z, self.h, self.offsets,
                                              self.ngmax, self.nb, self.cnt, m=self.m, rho=self.rho,
                                              params=self.params_list(params), stream=stream,
                                              tree=self._tree)
        return self._tree

    def run_plain(self, params=None, stream=None):
        """The plain path, set after set, one tree per set."""
        pl = self.params_list(params)
        g = self.ngmax
        for i, (a, b) in enumerate(zip(self.offsets[:-1], self.offsets[1:])):
            a, b = int(a), int(b)
            if b == a:
                continue
            p = pl[i]
            if (p.get("octree") or p.get("group_size") or p.get("find_compact") or p.get("pack_leaves")
                    or p.get("dim", 3) != 3):
                raise ValueError("the plain path takes bucket_size, alpha and beta only")
            t = btree_build(self.x[a:b], self.y[a:b], self.z[a:b], self.h[a:b],
                            bucket_size=p["bucket_size"], alpha=p["alpha"], beta=p["beta"],
                            stream=stream, tree=self._trees.get(i))
            self._trees[i] = t
            btree_find_neighbors_density(t, self.m[a:b], g, self.nb[a * g:b * g], self.cnt[a:b],
                                         self.rho[a:b], stream=stream)

    def results(self, i):
        """Host copies of set i's rows (capped), counts and densities."""
        a, b = int(self.offsets[i]), int(self.offsets[i + 1])
        nb = self.nb[a * self.ngmax:b * self.ngmax].view(-1, self.ngmax).cpu().numpy()
        cnt = self.cnt[a:b].cpu().numpy()
        rho = self.rho[a:b].cpu().numpy() if self.rho is not None else None
        return nb, cnt, rho

    def free(self):
        if self._tree is not None:
            self._tree.free()
            self._tree = None
        for t in self._trees.values():
            t.free()
        self._trees = {}


def shard_sets(sizes, world: int):
    """Assign sets to `world` ranks, largest first, each to the rank with the
    fewest particles so far (no data moves between ranks: sets are
    independent).  Returns one ascending list of set indices per rank."""
    world = int(world)
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    out = [[] for _ in range(world)]
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(i)
        load[r] += int(sizes[i])
    return [sorted(o) for o in out]


def list_checksum(nb, cnt, ngmax: int, chunk_rows: int = 1 << 17) -> int:
    """Order-sensitive checksum of the written part of every row (entries
    past min(count, ngmax) are unspecified and skipped).  Works in blocks of
    `chunk_rows` rows (a few hundred MB of temporaries) and reads the result
    back once."""
    import torch
    n = int(cnt.numel())
    total = torch.zeros((), dtype=torch.int64, device=nb.device)
    col = torch.arange(ngmax, device=nb.device, dtype=torch.int64)
    for a in range(0, n, chunk_rows):
        b = min(n, a + chunk_rows)
        rows = nb[a * ngmax:b * ngmax].view(-1, ngmax).to(torch.int64)
        used = col[None, :] < cnt[a:b].to(torch.int64).clamp(max=ngmax)[:, None]
        w = (torch.arange(a, b, device=nb.device, dtype=torch.int64)[:, None] * ngmax + col[None, :])
        w = w % 1000003 + 1
        total += torch.where(used, (rows + 7) * w, torch.zeros_like(rows)).sum()
    return int(total.item())
