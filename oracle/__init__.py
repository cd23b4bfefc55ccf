"""CPU oracle for the b-tree neighbour search -- TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 statement of the method of arXiv:1910.02639 (BuildTree,
Algorithm 1 / Eqs. 1-4; FindNeighbors, Algorithm 2 / Eqs. 5-6), plus the
brute-force O(n^2) definition of the neighbour lists and the FP64 M4 density.
The arithmetic lives in ``btree_oracle.c`` (compiled with gcc,
``-ffp-contract=off``); this module only marshals numpy arrays.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  It imports nothing from the CUDA library and the
library imports nothing from here.

Parity status per function (what pins it, see ``tests/test_oracle_pins.py``):
  branching_factor  -- closed form b^3 s >= n > (b-1)^3 s, perfect-cube trap.
  child_coord/id    -- the worked example of Sec. 3.1 (coords (7,8,1), j=187).
  cell_range        -- the 2D example of Fig. 1 (x cells 2..4, y cells 3..4).
  build             -- ratio loop collapses a clustered cell to b=2 (Sec. 3.1
                       step 3), invariants (each particle in one leaf, boxes tile);
                       octree mode: a 8x8x8 lattice at s=1 is the perfect
                       depth-3 octree (73 internal cells); k = 2: closed-form
                       b^2 s >= n, an 8x8 planar lattice gives the perfect
                       quadtree (21 internal cells) and z is never split.
  find_brute        -- closed-form lattice counts (92 interior neighbours at
                       h=1.5, strict <), hand-checked tiny sets, pair symmetry.
  find_tree         -- equal to find_brute (the definition) on random sets.
  m4/kernel_w       -- normalisation, continuity, central value 1/(pi h^3).
  density           -- isolated particle, lattice Riemann sum ~ 1.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "btree_oracle.c")
_LIB = os.path.join(_HERE, "_btree_oracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
          "-shared", "-std=gnu11"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no CUDA involved). Returns the .so path."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", *CFLAGS, "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
        lib.orc_branching_factor.restype = i64
        lib.orc_branching_factor.argtypes = [i64, i64]
        lib.orc_child_coord.restype = i64
        lib.orc_child_coord.argtypes = [dbl, dbl, dbl, i64]
        lib.orc_child_id.restype = i64
        lib.orc_child_id.argtypes = [i64, i64, i64, i64]
        lib.orc_cell_range.restype = None
        lib.orc_cell_range.argtypes = [dbl, dbl, dbl, dbl, i64,
                                       ctypes.POINTER(i64), ctypes.POINTER(i64)]
        lib.orc_distance2.restype = dbl
        lib.orc_distance2.argtypes = [ctypes.c_float] * 6
        lib.orc_radius2.restype = dbl
        lib.orc_radius2.argtypes = [ctypes.c_float]
        lib.orc_build.restype = vp
        lib.orc_build.argtypes = [vp, vp, vp, i64, i64, dbl, dbl]
        lib.orc_build2.restype = vp
        lib.orc_build2.argtypes = [vp, vp, vp, i64, i64, dbl, dbl, ctypes.c_int]
        lib.orc_build_ex.restype = vp
        lib.orc_build_ex.argtypes = [vp, vp, vp, i64, i64, dbl, dbl, ctypes.c_int, ctypes.c_int]
        lib.orc_branching_factor2.restype = i64
        lib.orc_branching_factor2.argtypes = [i64, i64]
        lib.orc_free.restype = None
        lib.orc_free.argtypes = [vp]
        for f in ("orc_num_nodes", "orc_num_slots"):
            getattr(lib, f).restype = i64
            getattr(lib, f).argtypes = [vp]
        for f in ("orc_max_depth", "orc_num_oversized"):
            getattr(lib, f).restype = i32
            getattr(lib, f).argtypes = [vp]
        lib.orc_export.restype = None
        lib.orc_export.argtypes = [vp] * 11
        lib.orc_find_tree.restype = None
        lib.orc_find_tree.argtypes = [vp, vp, i64, i64, i64, vp, vp]
        lib.orc_find_brute.restype = None
        lib.orc_find_brute.argtypes = [vp, vp, vp, vp, i64, i64, i64, i64, vp, vp]
        lib.orc_m4_shape.restype = dbl
        lib.orc_m4_shape.argtypes = [dbl]
        lib.orc_kernel_w.restype = dbl
        lib.orc_kernel_w.argtypes = [dbl, dbl]
        lib.orc_density.restype = None
        lib.orc_density.argtypes = [vp, vp, vp, i64, i64, vp]
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_num_threads.argtypes = []
        _lib = lib
        return lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


# ---------------------------------------------------------------- scalars
def branching_factor(n: int, s: int, k: int = 3) -> int:
    """Eq. 1 in exact integers (k = 3, or 2 for a two-dimensional tree)."""
    if k == 2:
        return int(_load().orc_branching_factor2(n, s))
    return int(_load().orc_branching_factor(n, s))


def child_coord(x: float, lo: float, hi: float, b: int) -> int:
    """Eq. 2 (clamped) in FP64."""
    return int(_load().orc_child_coord(x, lo, hi, b))


def child_id(c1: int, c2: int, c3: int, b: int) -> int:
    """Eq. 3."""
    return int(_load().orc_child_id(c1, c2, c3, b))


def cell_range(x: float, two_h: float, lo: float, hi: float, b: int):
    """Eqs. 5-6 for one dimension (with the outward safety margin)."""
    a, c = ctypes.c_int64(), ctypes.c_int64()
    _load().orc_cell_range(x, two_h, lo, hi, b, ctypes.byref(a), ctypes.byref(c))
    return int(a.value), int(c.value)


def distance2(pi, pj) -> float:
    """D = ((dx*dx + dy*dy) + dz*dz) in FP64 from float32 inputs."""
    pi = np.asarray(pi, dtype=np.float32)
    pj = np.asarray(pj, dtype=np.float32)
    return float(_load().orc_distance2(*map(float, pi), *map(float, pj)))


def radius2(h: float) -> float:
    return float(_load().orc_radius2(float(np.float32(h))))


def m4_shape(q: float) -> float:
    return float(_load().orc_m4_shape(q))


def kernel_w(r: float, h: float) -> float:
    return float(_load().orc_kernel_w(r, h))


def num_threads() -> int:
    return int(_load().orc_num_threads())


# ---------------------------------------------------------------- tree
class OracleTree:
    """The oracle's b-tree (Algorithm 1) over float32 positions."""

    def __init__(self, x, y, z, bucket_size=16, alpha=0.5, beta=0.5, octree=False, dim=3):
        lib = _load()
        self.x, self.y, self.z = _f32(x), _f32(y), _f32(z)
        self.n = int(self.x.shape[0])
        self.bucket_size = int(bucket_size)
        self.dim = int(dim)
        self._t = lib.orc_build_ex(_ptr(self.x), _ptr(self.y), _ptr(self.z), self.n,
                                   self.bucket_size, float(alpha), float(beta), int(bool(octree)),
                                   self.dim)
        if not self._t:
            raise ValueError("oracle build rejected its arguments")
        self._lib = lib

    def __del__(self):
        t = getattr(self, "_t", None)
        if t:
            self._lib.orc_free(t)
            self._t = None

    @property
    def num_nodes(self) -> int:
        return int(self._lib.orc_num_nodes(self._t))

    @property
    def max_depth(self) -> int:
        return int(self._lib.orc_max_depth(self._t))

    @property
    def num_oversized(self) -> int:
        return int(self._lib.orc_num_oversized(self._t))

    def export(self) -> dict:
        """Node table, child table and particle order as numpy arrays."""
        nn = self.num_nodes
        ns = int(self._lib.orc_num_slots(self._t))
        out = dict(
            lo=np.zeros((nn, 3)), hi=np.zeros((nn, 3)),
            start=np.zeros(nn, np.int64), count=np.zeros(nn, np.int64),
            depth=np.zeros(nn, np.int32), b=np.zeros(nn, np.int32),
            slot0=np.zeros(nn, np.int64), oversized=np.zeros(nn, np.int32),
            child=np.zeros(max(ns, 1), np.int64), perm=np.zeros(max(self.n, 1), np.int64))
        self._lib.orc_export(self._t, *[_ptr(out[k]) for k in (
            "lo", "hi", "start", "count", "depth", "b", "slot0", "oversized",
            "child", "perm")])
        out["child"] = out["child"][:ns]
        out["perm"] = out["perm"][:self.n]
        return out

    def find(self, h, ngmax, q0=0, q1=None):
        """Tree-walk lists (Algorithm 2) for queries [q0, q1)."""
        h = _f32(h)
        q1 = self.n if q1 is None else q1
        nq = max(q1 - q0, 0)
        nb = np.empty((nq, ngmax), np.int32)
        cnt = np.empty(nq, np.int32)
        if nq:
            self._lib.orc_find_tree(self._t, _ptr(h), q0, q1, ngmax, _ptr(nb), _ptr(cnt))
        return nb, cnt

    def density(self, h, m, q0=0, q1=None):
        """FP64 M4 density over the uncapped neighbour sets."""
        h, m = _f32(h), _f32(m)
        q1 = self.n if q1 is None else q1
        nq = max(q1 - q0, 0)
        rho = np.empty(nq, np.float64)
        if nq:
            self._lib.orc_density(self._t, _ptr(h), _ptr(m), q0, q1, _ptr(rho))
        return rho


def find_brute(x, y, z, h, ngmax, q0=0, q1=None):
    """O(n^2) lists: the definition N(i) = {j != i : D(i,j) < R(i)}."""
    x, y, z, h = _f32(x), _f32(y), _f32(z), _f32(h)
    n = int(x.shape[0])
    q1 = n if q1 is None else q1
    nq = max(q1 - q0, 0)
    nb = np.empty((nq, ngmax), np.int32)
    cnt = np.empty(nq, np.int32)
    if nq:
        _load().orc_find_brute(_ptr(x), _ptr(y), _ptr(z), _ptr(h), n, q0, q1, ngmax,
                               _ptr(nb), _ptr(cnt))
    return nb, cnt
