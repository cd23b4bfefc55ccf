"""One particle set split over several ranks: slabs along x plus one halo
exchange.

The paper builds and searches one tree per process (parallel over particles
within a node, Sec. 4) and leaves the split of one set over several nodes to
future work (Sec. 5).  Here the set is cut into slabs of equal particle count
along x; every rank receives, besides the particles of its own slab, the
particles of the other slabs that can be neighbours of its own ones (those
within R = 2 max(h) of its own particles' x-extent, R widened by 2^-20),
builds one tree over both and searches it.  A neighbour j of particle i satisfies D(i, j) <
(2 h_i)^2, hence |x_j - x_i| < 2 h_i (1 + 2^-53) (the binary64 square of the
exact float difference cannot exceed D), so it lies in the halo; and since
the local particles are kept in ascending global index, a row of local
indices maps to global indices without reordering.  Rows, counts and
densities are therefore those of a single run over the whole set, bit for bit
(the density of a particle is summed in the order of its list).

Data moves twice, both times as one all-to-all over the process group: the
particles to the rank that owns their slab, then the halo copies.  The
records travel as float64 rows (x, y, z, h, m exactly, the global index
exactly below 2^53) on the CPU for gloo and on the GPU for NCCL.
"""
from __future__ import annotations

import numpy as np

_HALO_SLACK = 1.0 + 2.0 ** -20
_SAMPLES_PER_RANK = 4096


def _exchange(dist, group, rows, dest, world, device):
    """Send rows[k] to rank dest[k]; returns the rows this rank receives
    (grouped by source rank, each group in its sender's order)."""
    import torch
    order = torch.argsort(dest, stable=True)
    rows = rows[order]
    send = torch.bincount(dest, minlength=world).to(torch.int64)
    r_dev = torch.empty(world, dtype=torch.int64, device=device)
    dist.all_to_all_single(r_dev, send.to(device), group=group)
    recv = r_dev.cpu()
    out = torch.empty((int(recv.sum()), rows.shape[1]), dtype=rows.dtype, device=device)
    dist.all_to_all_single(out, rows.to(device).contiguous(), output_split_sizes=recv.tolist(),
                           input_split_sizes=send.tolist(), group=group)
    return out


def slab_cuts(dist, group, x, world, device):
    """world - 1 cut positions along x giving slabs of about equal particle
    count, from an evenly strided sample of every rank's particles."""
    import torch
    n = int(x.numel())
    k = min(n, _SAMPLES_PER_RANK)
    idx = (torch.arange(k, dtype=torch.int64) * n) // max(k, 1)
    xs = torch.sort(x.cpu().to(torch.float64))[0]
    smp = torch.full((_SAMPLES_PER_RANK,), float("nan"), dtype=torch.float64)
    smp[:k] = xs[idx]
    allsmp = [torch.empty(_SAMPLES_PER_RANK, dtype=torch.float64, device=device) for _ in range(world)]
    dist.all_gather(allsmp, smp.to(device), group=group)
    v = torch.cat([a.cpu() for a in allsmp])
    v = torch.sort(v[~torch.isnan(v)])[0]
    if v.numel() == 0:
        return np.zeros(world - 1, np.float32)
    q = [(r * v.numel()) // world for r in range(1, world)]
    # cuts are floats: a particle belongs to slab r iff cut[r-1] <= x < cut[r]
    return np.array([np.float32(v[i].item()) for i in q], np.float32)


def _gpu_compute(x, y, z, h, m, ngmax, bucket_size, density):
    """Build + fused find (+ density) on the local particles, on their device."""
    import torch
    from . import btree_build, btree_find_neighbors, btree_find_neighbors_density
    n = int(x.numel())
    nb = torch.full((max(n, 1) * ngmax,), -1, dtype=torch.int32, device=x.device)
    cnt = torch.zeros(max(n, 1), dtype=torch.int32, device=x.device)
    rho = torch.zeros(max(n, 1), dtype=torch.float32, device=x.device) if density else None
    if n:
        tree = btree_build(x, y, z, h, bucket_size=bucket_size)
        if density:
            btree_find_neighbors_density(tree, m, ngmax, nb, cnt, rho)
        else:
            btree_find_neighbors(tree, ngmax, nb, cnt)
        torch.cuda.synchronize(x.device)
        tree.free()
    return nb.view(-1, ngmax)[:n], cnt[:n], (rho[:n] if density else None)


def decomposed_find(x, y, z, h, m, gidx, ngmax: int, group=None, bucket_size: int = 16,
                    density: bool = True, compute=None):
    """FindNeighbors (and the density) for one particle set spread over the
    ranks of `group`.

    x, y, z, h, m: float32 tensors of the particles this rank holds (any
    subset of the set; on the compute device), gidx: their int64 global
    indices.  Returns a dict for the particles this rank owns after the split
    (its slab of x), in ascending global index: ``gidx`` [k] int64, ``nb``
    [k, ngmax] int32 global neighbour indices (ascending, capped, -1 after
    the count), ``cnt`` [k] int32 (uncapped), ``rho`` [k] float32 (if
    `density`), plus ``halo`` (particles received as halo) and ``cuts``.

    `compute(x, y, z, h, m, ngmax, bucket_size, density) -> (nb, cnt, rho)`
    runs one set on the local particles (set-local indices); the default is
    this library's GPU build and fused find.
    """
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    device = torch.device("cuda", torch.cuda.current_device()) \
        if dist.get_backend(group) == "nccl" else torch.device("cpu")
    compute = compute or _gpu_compute
    dev = x.device

    # 1. slabs of equal count along x; every particle to its slab's rank
    cuts = slab_cuts(dist, group, x, world, device)
    xc = x.detach().cpu()
    owner = torch.from_numpy(np.searchsorted(cuts, xc.numpy(), side="right").astype(np.int64))
    rec = torch.stack([xc.double(), y.detach().cpu().double(), z.detach().cpu().double(),
                       h.detach().cpu().double(), m.detach().cpu().double(),
                       gidx.detach().cpu().double()], dim=1)
    own = _exchange(dist, group, rec, owner, world, device).cpu()

    # 2. halo: my particles within R_r of the x-extent of rank r's own
    # particles, for every r != me
    if own.shape[0]:
        ext = [float(own[:, 0].min()), float(own[:, 0].max()),
               float(own[:, 3].max()) * 2.0 * _HALO_SLACK]
    else:
        ext = [np.inf, -np.inf, 0.0]
    allext = [torch.empty(3, dtype=torch.float64, device=device) for _ in range(world)]
    dist.all_gather(allext, torch.tensor(ext, dtype=torch.float64, device=device), group=group)
    allext = [v.cpu().tolist() for v in allext]
    ox = own[:, 0]
    rows, dest = [], []
    for r in range(world):
        if r == rank:
            continue
        xlo, xhi, rr = allext[r]
        sel = (ox >= xlo - rr) & (ox <= xhi + rr)
        rows.append(own[sel])
        dest.append(torch.full((int(sel.sum()),), r, dtype=torch.int64))
    send = torch.cat(rows) if rows else own[:0]
    dst = torch.cat(dest) if dest else torch.zeros(0, dtype=torch.int64)
    halo = _exchange(dist, group, send, dst, world, device).cpu()

    # 3. one set over own + halo particles, in ascending global index
    loc = torch.cat([own, halo])
    gl = loc[:, 5].to(torch.int64)
    order = torch.argsort(gl)
    loc, gl = loc[order], gl[order]
    is_own = torch.zeros(loc.shape[0], dtype=torch.bool)
    is_own[:own.shape[0]] = True
    is_own = is_own[order]
    f = lambda c: loc[:, c].to(torch.float32).to(dev).contiguous()
    nb, cnt, rho = compute(f(0), f(1), f(2), f(3), f(4), ngmax, bucket_size, density)
    nb, cnt = nb.cpu(), cnt.cpu()
    k = is_own.nonzero().flatten()
    nb, cnt = nb[k], cnt[k]
    valid = torch.arange(ngmax).unsqueeze(0) < cnt.clamp(max=ngmax).unsqueeze(1)
    nbg = torch.where(valid, gl[nb.clamp(min=0).to(torch.int64)].to(torch.int32),
                      torch.full_like(nb, -1))
    out = dict(gidx=gl[k], nb=nbg, cnt=cnt, halo=int(halo.shape[0]), cuts=cuts)
    if density:
        out["rho"] = rho.cpu()[k]
    return out
