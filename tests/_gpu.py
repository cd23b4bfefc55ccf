"""Helpers for the GPU parity tests: run the CUDA path through the C ABI and
compare with the oracle."""
from __future__ import annotations

import numpy as np


def to_dev(s, dev="cuda:0"):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    return t(s.x), t(s.y), t(s.z), t(s.h), t(s.m)


def run_gpu(s, bucket_size=16, ngmax=256, alpha=0.5, beta=0.5, density=False, tree=None):
    """Build + find (+ fused density).  Rows are pre-filled with -1 so that
    full rows compare with the oracle's convention."""
    import torch
    import paper_1910_02639_gb300 as bt
    x, y, z, h, m = to_dev(s)
    tree = bt.btree_build(x, y, z, h, bucket_size=bucket_size, alpha=alpha, beta=beta, tree=tree)
    nb = torch.full((max(s.n, 1) * ngmax,), -1, dtype=torch.int32, device=x.device)
    cnt = torch.full((max(s.n, 1),), -7, dtype=torch.int32, device=x.device)
    rho = None
    if density:
        rho = torch.empty(max(s.n, 1), dtype=torch.float32, device=x.device)
        bt.btree_find_neighbors_density(tree, m, ngmax, nb, cnt, rho)
    else:
        bt.btree_find_neighbors(tree, ngmax, nb, cnt)
    torch.cuda.synchronize()
    out = dict(tree=tree, nb_dev=nb, cnt_dev=cnt, rho_dev=rho,
               nb=nb.view(-1, ngmax)[:s.n].cpu().numpy(), cnt=cnt[:s.n].cpu().numpy())
    if density:
        out["rho"] = rho[:s.n].cpu().numpy()
    return out


def canonical_tree_gpu(e, n, root=0, off=0, k=3):
    """Per-internal-cell table and per-particle (cell, sub-cell id) from the
    GPU export; `root` is the set's root node, `off` its first particle."""
    return _canon(e["lo"], e["hi"], e["depth"], e["b"], e["count"],
                  lambda i: _gpu_children(e, i, off, k), n, root)


def _gpu_children(e, i, off=0, k=3):
    b = int(e["b"][i])
    k0 = int(e["slot0"][i])
    out = []
    for j in range(b ** k):
        c = int(e["slot_child"][k0 + j])
        st, ct = int(e["slot_start"][k0 + j]), int(e["slot_count"][k0 + j])
        if c >= 0 and int(e["b"][c]) > 0:
            out.append((j, ("node", c)))
        else:
            out.append((j, ("leaf", e["order"][st:st + ct] - off)))
    return out


def canonical_tree_oracle(e, n, k=3):
    return _canon(e["lo"], e["hi"], e["depth"], e["b"], e["count"],
                  lambda i: _orc_children(e, i, k), n)


def _orc_children(e, i, k=3):
    b = int(e["b"][i])
    k0 = int(e["slot0"][i])
    out = []
    for j in range(b ** k):
        c = int(e["child"][k0 + j])
        if int(e["b"][c]) > 0:
            out.append((j, ("node", c)))
        else:
            st, ct = int(e["start"][c]), int(e["count"][c])
            out.append((j, ("leaf", e["perm"][st:st + ct])))
    return out


def _canon(lo, hi, depth, b, count, children, n, root=0):
    """Walk from the root: cells keyed by (depth, lo, hi); for each internal
    cell its b and count; for each particle the key of its parent cell and its
    sub-cell id."""
    cells = {}
    pcell = np.full(n, -1, np.int64)
    pj = np.full(n, -1, np.int64)
    keys = []
    stack = [root]
    if n == 0:
        return cells, pcell, pj, keys
    if int(b[root]) == 0:
        keys.append(("leafroot",))
        pcell[:] = 0
        pj[:] = 0
        return cells, pcell, pj, keys
    while stack:
        i = stack.pop()
        key = (int(depth[i]), tuple(lo[i]), tuple(hi[i]))
        ki = len(keys)
        keys.append(key)
        cells[key] = (int(b[i]), int(count[i]))
        for j, (kind, v) in children(i):
            if kind == "node":
                stack.append(v)
            else:
                pcell[v] = ki
                pj[v] = j
    return cells, pcell, pj, keys


def compare_trees(gpu_export, orc_export, n, root=0, off=0, k=3):
    gc, gp, gj, gk = canonical_tree_gpu(gpu_export, n, root, off, k)
    oc, op_, oj, ok = canonical_tree_oracle(orc_export, n, k)
    assert gc == oc, "internal cells (depth, box, b, count) differ"
    # map cell indices through their keys
    gkey = np.array([hash(k) for k in gk] + [0], dtype=np.int64)
    okey = np.array([hash(k) for k in ok] + [0], dtype=np.int64)
    assert np.array_equal(gkey[gp], okey[op_]), "leaf parent cells differ"
    assert np.array_equal(gj, oj), "leaf sub-cell ids differ"
