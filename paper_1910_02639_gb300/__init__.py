"""GB300 b-tree neighbour search (arXiv:1910.02639) -- Python binding.

A thin ctypes layer over the C ABI of ``libbtree.so`` (``include/btree.h``):
the same function names, argument marshalling only.  Every step of the build,
the search and the density sum runs in the library's CUDA kernels; there is
no CPU fallback.  Importing the package does not load the library; the first
call does, and raises if it was not built (``python -m
paper_1910_02639_gb300.build_ext`` or ``__graft_entry__.build()``).

Tensors are PyTorch CUDA tensors (device memory and streams only):
positions and smoothing lengths float32 [n], contiguous.
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = [
    "BtreeError", "Tree", "btree_build", "btree_build_batched", "btree_build_find_batched",
    "btree_find_neighbors", "btree_find_neighbors_csr", "btree_pack_rows",
    "btree_find_neighbors_density", "btree_find_neighbors_density_noalloc",
    "btree_noalloc_max_particles", "sph_density", "btree_status", "btree_get_info",
    "btree_export", "btree_free", "btree_strerror", "btree_version", "btree_kernel_launches",
    "btree_arith_rates", "Allocator", "torch_allocator",
    "library_path",
    "BT_OK", "BT_WARN_NGMAX", "BT_WARN_OVERSIZED_LEAF",
]

BT_OK = 0
BT_ERR_ARG = -1
BT_ERR_OOM = -2
BT_ERR_CUDA = -3
BT_ERR_TIMEOUT = -4
BT_ERR_NONFINITE = -5
BT_ERR_CAPACITY = -6
BT_WARN_NGMAX = 1
BT_WARN_OVERSIZED_LEAF = 2

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libbtree.so")
_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _LIB_PATH


class BtreeError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {btree_strerror(status)} ({status})")


class _Info(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("bucket_size", ctypes.c_int32),
                ("max_depth", ctypes.c_int32), ("num_nodes", ctypes.c_int64),
                ("num_slots", ctypes.c_int64), ("num_groups", ctypes.c_int64),
                ("root_b", ctypes.c_int32), ("num_oversized", ctypes.c_int32),
                ("build_ms", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(
                f"{_LIB_PATH} is missing: build the CUDA library first "
                "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(_LIB_PATH)
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.btree_build.restype = ctypes.c_int
        lib.btree_build.argtypes = [vp, vp, vp, vp, i64, ctypes.c_int, dbl, dbl, vp, vp,
                                    ctypes.POINTER(vp)]
        lib.btree_build_batched.restype = ctypes.c_int
        lib.btree_build_batched.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int, vp, vp, vp,
                                            ctypes.POINTER(vp)]
        lib.btree_build_find_batched.restype = ctypes.c_int
        lib.btree_build_find_batched.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_int, vp,
                                                 ctypes.c_int, vp, vp, vp, vp, vp,
                                                 ctypes.POINTER(vp)]
        lib.btree_find_neighbors_csr.restype = ctypes.c_int
        lib.btree_find_neighbors_csr.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, ctypes.c_int64,
                                                 ctypes.POINTER(ctypes.c_int64), vp]
        lib.btree_pack_rows.restype = ctypes.c_int
        lib.btree_pack_rows.argtypes = [vp, vp, vp, ctypes.c_int, vp, vp, ctypes.c_int64,
                                        ctypes.POINTER(ctypes.c_int64), vp]
        lib.btree_find_neighbors.restype = ctypes.c_int
        lib.btree_find_neighbors.argtypes = [vp, ctypes.c_int, vp, vp, vp]
        lib.btree_find_neighbors_density.restype = ctypes.c_int
        lib.btree_find_neighbors_density.argtypes = [vp, vp, ctypes.c_int, vp, vp, vp, vp]
        lib.btree_find_neighbors_density_noalloc.restype = ctypes.c_int
        lib.btree_find_neighbors_density_noalloc.argtypes = [vp, vp, ctypes.c_int, vp, vp, vp, vp]
        lib.btree_noalloc_max_particles.restype = ctypes.c_int64
        lib.btree_noalloc_max_particles.argtypes = []
        lib.sph_density.restype = ctypes.c_int
        lib.sph_density.argtypes = [vp, vp, vp, vp, ctypes.c_int, vp, vp]
        lib.btree_status.restype = ctypes.c_int
        lib.btree_status.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int)]
        lib.btree_get_info.restype = ctypes.c_int
        lib.btree_get_info.argtypes = [vp, ctypes.POINTER(_Info)]
        lib.btree_export.restype = ctypes.c_int
        lib.btree_export.argtypes = [vp, vp] + [vp] * 11
        lib.btree_free.restype = None
        lib.btree_free.argtypes = [vp]
        lib.btree_strerror.restype = ctypes.c_char_p
        lib.btree_strerror.argtypes = [ctypes.c_int]
        lib.btree_version.restype = ctypes.c_char_p
        lib.btree_version.argtypes = []
        lib.btree_kernel_launches.restype = ctypes.c_uint64
        lib.btree_kernel_launches.argtypes = []
        lib.btree_arith_rates.restype = ctypes.c_int
        lib.btree_arith_rates.argtypes = [vp, ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                                          ctypes.POINTER(dbl)]
        _lib = lib
        return lib


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t, dtype, what, numel=None):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if numel is not None and t.numel() < numel:
        raise ValueError(f"{what} has {t.numel()} elements, needs {numel}")
    return ctypes.c_void_p(t.data_ptr())


def _check(status: int, what: str) -> int:
    if status < 0:
        raise BtreeError(status, what)
    return status


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class _CAllocator(ctypes.Structure):
    _fields_ = [("ctx", ctypes.c_void_p), ("alloc", _ALLOC_FN), ("free", _FREE_FN)]


class Allocator:
    """A bt_allocator (include/btree.h) from two Python callables:
    ``alloc(nbytes, stream) -> device address`` (an int; 0 or None when out
    of memory) and ``free(address, stream)``; ``stream`` is the cudaStream_t
    as an int.  A tree built with it takes every internal buffer from it and
    returns them through it when freed.  The callbacks must not raise."""

    def __init__(self, alloc, free):
        def _a(ctx, nbytes, stream):
            try:
                p = alloc(int(nbytes), int(stream or 0))
            except Exception:
                p = 0
            return int(p) if p else None

        def _f(ctx, ptr, stream):
            try:
                free(int(ptr or 0), int(stream or 0))
            except Exception:
                pass

        self._a, self._f = _ALLOC_FN(_a), _FREE_FN(_f)  # kept alive with the allocator
        self.c = _CAllocator(None, self._a, self._f)


def torch_allocator(device=None) -> Allocator:
    """PyTorch's caching allocator behind a tree's buffers (stream-ordered
    reuse on the stream the library passes)."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    return Allocator(lambda n, st: torch.cuda.caching_allocator_alloc(n, dev, st),
                     lambda p, st: torch.cuda.caching_allocator_delete(p))


class Tree:
    """Owns one btree_t.  Keeps the last build status in ``status``."""

    def __init__(self):
        self._ptr = ctypes.c_void_p(None)
        self.status = BT_OK
        self.n = 0
        self._allocator = None  # keeps an Allocator's callbacks alive until free()

    @property
    def handle(self):
        return self._ptr

    def free(self):
        if self._ptr and self._ptr.value:
            _load().btree_free(self._ptr)
        self._ptr = ctypes.c_void_p(None)
        self._allocator = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def info(self) -> dict:
        return btree_get_info(self)


def btree_build(x, y, z, h, bucket_size: int = 16, alpha: float = 0.5, beta: float = 0.5,
                stream=None, tree: Tree | None = None, allocator: Allocator | None = None) -> Tree:
    """BuildTree (Algorithm 1).  Rebuilds `tree` in place when given.  With
    `allocator` the tree's buffers come from it (else cudaMallocAsync)."""
    import torch
    lib = _load()
    n = int(x.numel())
    ptrs = [_dptr(a, torch.float32, nm, n) for a, nm in ((x, "x"), (y, "y"), (z, "z"), (h, "h"))]
    t = tree if tree is not None else Tree()
    if allocator is not None:
        t._allocator = allocator
    st = lib.btree_build(*ptrs, n, int(bucket_size), float(alpha), float(beta),
                         ctypes.byref(allocator.c) if allocator is not None else None,
                         ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(t._ptr))
    _check(st, "btree_build")
    t.status = st
    t.n = n
    return t


BT_SET_OCTREE = 1
BT_SET_FIND_COMPACT = 2
BT_SET_2D = 4
BT_SET_PACK_LEAVES = 8


class _SetParams(ctypes.Structure):
    _fields_ = [("bucket_size", ctypes.c_int), ("flags", ctypes.c_int),
                ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("group_size", ctypes.c_int), ("reserved", ctypes.c_int)]


def _set_params(params, nsets):
    if params is None:
        return None
    plist = [params] * nsets if isinstance(params, dict) else list(params)
    if len(plist) != nsets:
        raise ValueError("one parameter dict per set")
    c_par = (_SetParams * nsets)()
    for i, p in enumerate(plist):
        c_par[i].bucket_size = int(p.get("bucket_size", 16))
        c_par[i].flags = ((BT_SET_OCTREE if p.get("octree", False) else 0) |
                          (BT_SET_FIND_COMPACT if p.get("find_compact", False) else 0) |
                          (BT_SET_2D if int(p.get("dim", 3)) == 2 else 0) |
                          (BT_SET_PACK_LEAVES if p.get("pack_leaves", False) else 0))
        c_par[i].alpha = float(p.get("alpha", 0.5))
        c_par[i].beta = float(p.get("beta", 0.5))
        c_par[i].group_size = int(p.get("group_size", 0))
    return c_par


def btree_build_batched(x, y, z, h, offsets, params=None, stream=None,
                        tree: Tree | None = None) -> Tree:
    """BuildTree for many sets at once.  x, y, z, h: the sets concatenated;
    offsets: nsets+1 ints; params: per-set dicts with bucket_size, alpha,
    beta, octree, group_size (or one dict for all, or None for the
    defaults)."""
    import torch
    lib = _load()
    n = int(x.numel())
    offs = [int(v) for v in offsets]
    nsets = len(offs) - 1
    if nsets < 1 or offs[0] != 0 or offs[-1] != n:
        raise ValueError("offsets must run from 0 to the number of particles")
    ptrs = [_dptr(a, torch.float32, nm, n) for a, nm in ((x, "x"), (y, "y"), (z, "z"), (h, "h"))]
    c_offs = (ctypes.c_int64 * (nsets + 1))(*offs)
    c_par = _set_params(params, nsets)
    t = tree if tree is not None else Tree()
    st = lib.btree_build_batched(*ptrs, c_offs, nsets, c_par, None,
                                 ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(t._ptr))
    _check(st, "btree_build_batched")
    t.status = st
    t.n = n
    return t


def btree_build_find_batched(x, y, z, h, offsets, ngmax: int, neighbors, counts, m=None, rho=None,
                             params=None, stream=None, tree: Tree | None = None) -> Tree:
    """Batched build + find (+ density when m and rho are given) as one CUDA
    graph launch; synchronous.  Arguments as btree_build_batched and
    btree_find_neighbors_density."""
    import torch
    lib = _load()
    n = int(x.numel())
    offs = [int(v) for v in offsets]
    nsets = len(offs) - 1
    if nsets < 1 or offs[0] != 0 or offs[-1] != n:
        raise ValueError("offsets must run from 0 to the number of particles")
    ptrs = [_dptr(a, torch.float32, nm, n) for a, nm in ((x, "x"), (y, "y"), (z, "z"), (h, "h"))]
    if (m is None) != (rho is None):
        raise ValueError("give both m and rho, or neither")
    pm = _dptr(m, torch.float32, "m", n) if m is not None else None
    prho = _dptr(rho, torch.float32, "rho", n) if rho is not None else None
    pnb = _dptr(neighbors, torch.int32, "neighbors", n * ngmax)
    pc = _dptr(counts, torch.int32, "counts", n)
    c_offs = (ctypes.c_int64 * (nsets + 1))(*offs)
    c_par = _set_params(params, nsets)
    t = tree if tree is not None else Tree()
    st = lib.btree_build_find_batched(*ptrs, pm, c_offs, nsets, c_par, int(ngmax), pnb, pc, prho,
                                      None, ctypes.c_void_p(_stream_ptr(stream)),
                                      ctypes.byref(t._ptr))
    _check(st, "btree_build_find_batched")
    t.status = st
    t.n = n
    return t


BT_FIND_HALF = 1


def btree_find_neighbors_csr(tree: Tree, offsets, neighbors=None, m=None, rho=None,
                             stream=None, half: bool = False) -> int:
    """Compressed rows: offsets (int64 [n+1]) always written; rows written
    into `neighbors` (int32, any size >= the total) when given.  Returns the
    total number of pairs.  With neighbors=None only the offsets (and the
    density, when m and rho are given) are computed."""
    import torch
    lib = _load()
    n = tree.n
    if (m is None) != (rho is None):
        raise ValueError("give both m and rho, or neither")
    po = _dptr(offsets, torch.int64, "offsets", n + 1)
    pm = _dptr(m, torch.float32, "m", n) if m is not None else None
    pr = _dptr(rho, torch.float32, "rho", n) if rho is not None else None
    pn = _dptr(neighbors, torch.int32, "neighbors") if neighbors is not None else None
    cap = int(neighbors.numel()) if neighbors is not None else 0
    tot = ctypes.c_int64(0)
    st = lib.btree_find_neighbors_csr(tree.handle, BT_FIND_HALF if half else 0, pm, pr, po, pn, cap,
                                      ctypes.byref(tot),
                                      ctypes.c_void_p(_stream_ptr(stream)))
    _check(st, "btree_find_neighbors_csr")
    return int(tot.value)


def btree_pack_rows(tree: Tree, rows, counts, ngmax: int, offsets, csr=None, stream=None) -> int:
    """Pack fixed rows into compressed rows; returns the total entries."""
    import torch
    lib = _load()
    n = tree.n
    pr = _dptr(rows, torch.int32, "rows", n * ngmax)
    pc = _dptr(counts, torch.int32, "counts", n)
    po = _dptr(offsets, torch.int64, "offsets", n + 1)
    pcsr = _dptr(csr, torch.int32, "csr") if csr is not None else None
    cap = int(csr.numel()) if csr is not None else 0
    tot = ctypes.c_int64(0)
    st = lib.btree_pack_rows(tree.handle, pr, pc, int(ngmax), po, pcsr, cap, ctypes.byref(tot),
                             ctypes.c_void_p(_stream_ptr(stream)))
    _check(st, "btree_pack_rows")
    return int(tot.value)


def btree_find_neighbors(tree: Tree, ngmax: int, neighbors, counts, stream=None) -> int:
    """FindNeighbors (Algorithm 2): rows ascending by original index, capped."""
    import torch
    n = tree.n
    st = _load().btree_find_neighbors(
        tree.handle, int(ngmax), _dptr(neighbors, torch.int32, "neighbors", n * ngmax),
        _dptr(counts, torch.int32, "counts", n), ctypes.c_void_p(_stream_ptr(stream)))
    return _check(st, "btree_find_neighbors")


def btree_find_neighbors_density(tree: Tree, m, ngmax: int, neighbors, counts, rho,
                                 stream=None) -> int:
    """FindNeighbors fused with the M4 SPH density over the uncapped sets."""
    import torch
    n = tree.n
    st = _load().btree_find_neighbors_density(
        tree.handle, _dptr(m, torch.float32, "m", n), int(ngmax),
        _dptr(neighbors, torch.int32, "neighbors", n * ngmax),
        _dptr(counts, torch.int32, "counts", n), _dptr(rho, torch.float32, "rho", n),
        ctypes.c_void_p(_stream_ptr(stream)))
    return _check(st, "btree_find_neighbors_density")


def btree_find_neighbors_density_noalloc(tree: Tree, m, ngmax: int, neighbors, counts, rho,
                                         stream=None) -> int:
    """As btree_find_neighbors_density, for callers that cannot allocate
    device memory when they search: the library's only scratch buffer for
    this call is a fixed array compiled into it (trees of at most
    btree_noalloc_max_particles() particles; concurrent calls race on it)."""
    import torch
    n = tree.n
    st = _load().btree_find_neighbors_density_noalloc(
        tree.handle, _dptr(m, torch.float32, "m", n), int(ngmax),
        _dptr(neighbors, torch.int32, "neighbors", n * ngmax),
        _dptr(counts, torch.int32, "counts", n), _dptr(rho, torch.float32, "rho", n),
        ctypes.c_void_p(_stream_ptr(stream)))
    return _check(st, "btree_find_neighbors_density_noalloc")


def btree_noalloc_max_particles() -> int:
    return int(_load().btree_noalloc_max_particles())


def sph_density(tree: Tree, m, neighbors, counts, ngmax: int, rho, stream=None) -> int:
    """M4 density from existing rows (first min(count, ngmax) entries)."""
    import torch
    n = tree.n
    st = _load().sph_density(
        tree.handle, _dptr(m, torch.float32, "m", n),
        _dptr(neighbors, torch.int32, "neighbors", n * ngmax),
        _dptr(counts, torch.int32, "counts", n), int(ngmax),
        _dptr(rho, torch.float32, "rho", n), ctypes.c_void_p(_stream_ptr(stream)))
    return _check(st, "sph_density")


def btree_status(tree: Tree, stream=None) -> int:
    out = ctypes.c_int(0)
    _check(_load().btree_status(tree.handle, ctypes.c_void_p(_stream_ptr(stream)),
                                ctypes.byref(out)), "btree_status")
    return int(out.value)


def btree_get_info(tree: Tree) -> dict:
    info = _Info()
    _check(_load().btree_get_info(tree.handle, ctypes.byref(info)), "btree_get_info")
    return {k: getattr(info, k) for k, _ in _Info._fields_}


def btree_export(tree: Tree, stream=None) -> dict:
    """Copy the tree to host numpy arrays (node table, sub-cells, order)."""
    import numpy as np
    info = btree_get_info(tree)
    nn, ns, n = info["num_nodes"], info["num_slots"], info["n"]
    out = dict(lo=np.zeros((nn, 3)), hi=np.zeros((nn, 3)), b=np.zeros(nn, np.int32),
               depth=np.zeros(nn, np.int32), start=np.zeros(nn, np.int32),
               count=np.zeros(nn, np.int32), slot0=np.zeros(nn, np.int32),
               slot_start=np.zeros(ns, np.int32), slot_count=np.zeros(ns, np.int32),
               slot_child=np.zeros(ns, np.int32), order=np.zeros(n, np.int32))
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    st = _load().btree_export(tree.handle, ctypes.c_void_p(_stream_ptr(stream)),
                              p(out["lo"]), p(out["hi"]), p(out["b"]), p(out["depth"]),
                              p(out["start"]), p(out["count"]), p(out["slot0"]),
                              p(out["slot_start"]), p(out["slot_count"]),
                              p(out["slot_child"]), p(out["order"]))
    _check(st, "btree_export")
    return out


def btree_free(tree: Tree) -> None:
    tree.free()


def btree_strerror(status: int) -> str:
    return _load().btree_strerror(int(status)).decode()


def btree_version() -> str:
    return _load().btree_version().decode()


def btree_kernel_launches() -> int:
    """CUDA kernels launched by the library so far in this process."""
    return int(_load().btree_kernel_launches())


def btree_arith_rates(stream=None) -> dict:
    """Measured FMA throughput of the current device in GFLOP/s: scalar FP32,
    packed FP32x2 and binary64 (see btree.h)."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_load().btree_arith_rates(ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(a),
                                     ctypes.byref(b), ctypes.byref(c)), "btree_arith_rates")
    return {"fp32_gflops": a.value, "fp32x2_gflops": b.value, "fp64_gflops": c.value}
