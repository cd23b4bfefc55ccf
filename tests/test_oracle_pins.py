"""Pins for the CPU oracle: each check ties it to something other than itself --
values printed in the paper, closed forms, exact integer enumeration, textbook
properties of the M4 spline, brute force on tiny inputs."""
import itertools
import json
import math
import os

import numpy as np
import pytest

from paper_1910_02639_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# --------------------------------------------------------------- Eqs. 2-3
def test_worked_example_eq2_eq3(oracle):
    g = _golden("worked_example_eq2_eq3.json")
    for as_float in (False, True):
        xs = [float(np.float32(v)) if as_float else v for v in g["x"]]
        c = [oracle.child_coord(xs[l], g["box_lo"][l], g["box_hi"][l], g["b"]) for l in range(3)]
        assert c == g["coords"]
        assert oracle.child_id(*c, g["b"]) == g["id"]
    assert g["b"] ** 3 == g["num_subcells"]


def test_child_coord_clamps_and_degenerate(oracle):
    # particle exactly on the upper bound maps to the last cell, not cell b
    assert oracle.child_coord(5.0, 0.0, 5.0, 10) == 9
    assert oracle.child_coord(0.0, 0.0, 5.0, 10) == 0
    # slightly outside (rounding) is clamped
    assert oracle.child_coord(-1e-9, 0.0, 5.0, 10) == 0
    assert oracle.child_coord(5.0 + 1e-9, 0.0, 5.0, 10) == 9
    # zero-width dimension: every particle at coordinate 0
    assert oracle.child_coord(2.0, 2.0, 2.0, 7) == 0
    # Eq. 3 ordering: x fastest
    assert oracle.child_id(1, 0, 0, 4) == 1
    assert oracle.child_id(0, 1, 0, 4) == 4
    assert oracle.child_id(0, 0, 1, 4) == 16


# --------------------------------------------------------------- Eqs. 5-6
def test_fig1_range(oracle):
    g = _golden("fig1_range.json")
    rx = oracle.cell_range(g["particle"][0], g["two_h"], g["box_lo"][0], g["box_hi"][0], g["b"])
    ry = oracle.cell_range(g["particle"][1], g["two_h"], g["box_lo"][1], g["box_hi"][1], g["b"])
    assert list(rx) == g["x_cells"]
    assert list(ry) == g["y_cells"]


def test_cell_range_clamped(oracle):
    assert oracle.cell_range(0.1, 5.0, 0.0, 1.0, 4) == (0, 3)
    assert oracle.cell_range(0.5, 0.01, 0.0, 1.0, 4) == (1, 2)  # 0.5 is a boundary
    assert oracle.cell_range(0.3, 0.01, 0.0, 0.0, 4) == (0, 0)


# --------------------------------------------------------------- Eq. 1
def _icbrt_ceil(v: int) -> int:
    """ceil(v^(1/3)) for integers, by exact integer arithmetic."""
    r = int(round(v ** (1.0 / 3.0)))
    while r ** 3 < v:
        r += 1
    while r > 0 and (r - 1) ** 3 >= v:
        r -= 1
    return r


def test_branching_factor_values(oracle):
    # values at the workload sizes; n=1e6, s=8 is an exact cube (50^3 * 8)
    assert oracle.branching_factor(32768, 16) == 13
    assert oracle.branching_factor(10_000_000, 16) == 86
    assert oracle.branching_factor(10_000_000, 8) == 108
    assert oracle.branching_factor(1_000_000, 8) == 50
    assert oracle.branching_factor(17, 16) == 2


def test_branching_factor_closed_form(oracle):
    rng = np.random.default_rng(5)
    for _ in range(300):
        s = int(rng.integers(1, 65))
        n = int(rng.integers(s + 1, 50_000_000))
        b = oracle.branching_factor(n, s)
        # ceil of a rational cube root: b = ceil(cbrt(ceil(n/s)))
        assert b == max(2, _icbrt_ceil(-(-n // s)))


# --------------------------------------------------------------- Eq. 4
def test_ratio_loop_collapses_clustered_cell_to_octree(oracle):
    # 64 particles crowded into one corner of a box set by one far particle:
    # b0 = 3, 26 of 27 cells hold <= alpha*s particles -> halve to b = 2.
    rng = np.random.default_rng(1)
    p = rng.random((64, 3)).astype(np.float32) * np.float32(0.01)
    p = np.vstack([p, np.ones((1, 3), np.float32)])
    t = oracle.OracleTree(p[:, 0], p[:, 1], p[:, 2], bucket_size=4, alpha=0.5, beta=0.5)
    e = t.export()
    assert oracle.branching_factor(65, 4) == 3
    assert e["b"][0] == 2


def test_ratio_loop_keeps_b0_on_uniform_data(oracle):
    s = wl.uniform_cube(32768, seed=1911)
    t = oracle.OracleTree(s.x, s.y, s.z, bucket_size=16)
    e = t.export()
    assert e["b"][0] == 13
    assert t.max_depth <= 2


def test_beta_one_never_halves_and_beta_zero_always_halves(oracle):
    rng = np.random.default_rng(2)
    p = rng.random((3, 5000)).astype(np.float32) ** 3  # non-uniform
    t1 = oracle.OracleTree(p[0], p[1], p[2], bucket_size=8, alpha=0.5, beta=1.0)
    assert t1.export()["b"][0] == oracle.branching_factor(5000, 8)
    t0 = oracle.OracleTree(p[0], p[1], p[2], bucket_size=8, alpha=0.5, beta=0.0)
    b = t0.export()["b"]
    assert np.all(b[b > 0] == 2)  # every internal node collapses to an octree split


def _checkerboard_cells(drop=0):
    """One particle at the centre of each sub-cell (x+y+z even) of a 4x4x4
    grid: 32 occupied, 32 empty, and 0 and 3 occur in every dimension, so the
    bounding box maps the centres onto exactly these sub-cells (Eq. 2).
    `drop` removes that many occupied cells that do not set the box."""
    c = [(i, j, k) for k in range(4) for j in range(4) for i in range(4) if (i + j + k) % 2 == 0]
    keep = [t for t in c if 0 in t or 3 in t]
    inner = [t for t in c if t not in keep]
    c = keep + inner[:len(inner) - drop] if drop else c
    p = np.array(c, np.float32) + np.float32(0.5)
    return p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy()


def test_ratio_tie_accepts(oracle):
    # Eq. 4 at equality.  s = 1, alpha = 0.5: a sub-cell is underfull iff it is
    # empty.  32 particles: b0 = 4 (27 < 32 <= 64), 32 of the 64 sub-cells
    # empty, u = 32 = beta * b^3 exactly: r is not larger than beta, so b = 4
    # is kept (Sec. 3.1, step 3: halve only while r exceeds beta).
    x, y, z = _checkerboard_cells()
    assert x.shape[0] == 32 and oracle.branching_factor(32, 1) == 4
    e = oracle.OracleTree(x, y, z, bucket_size=1, alpha=0.5, beta=0.5).export()
    assert e["b"][0] == 4
    # every occupied sub-cell holds one particle: a leaf, no deeper node
    assert np.count_nonzero(e["b"]) == 1


def test_ratio_one_past_tie_halves(oracle):
    # the same grid with two inner occupied cells removed: 30 particles,
    # b0 = 4 still (27 < 30), u = 34 > 32: halve to b = 2.
    x, y, z = _checkerboard_cells(drop=2)
    assert x.shape[0] == 30 and oracle.branching_factor(30, 1) == 4
    e = oracle.OracleTree(x, y, z, bucket_size=1, alpha=0.5, beta=0.5).export()
    assert e["b"][0] == 2


# --------------------------------------------------------------- tree invariants
def _check_tree_invariants(e, n, s, k=3):
    leaf = e["b"] == 0
    # every particle in exactly one leaf
    seen = np.zeros(n, np.int64)
    for i in np.nonzero(leaf)[0]:
        seen[e["perm"][e["start"][i]:e["start"][i] + e["count"][i]]] += 1
    assert np.all(seen == 1)
    assert e["count"][leaf].sum() == n
    # leaves hold at most s particles unless flagged oversized
    assert np.all((e["count"][leaf] <= s) | (e["oversized"][leaf] == 1))
    # children tile the parent: counts add up, boxes inside the parent box
    for i in np.nonzero(~leaf)[0]:
        b = int(e["b"][i])
        ch = e["child"][e["slot0"][i]:e["slot0"][i] + b ** k]
        assert e["count"][ch].sum() == e["count"][i]
        assert np.all(e["lo"][ch] >= e["lo"][i]) and np.all(e["hi"][ch] <= e["hi"][i])
        assert np.all(e["depth"][ch] == e["depth"][i] + 1)
        assert np.all(e["start"][ch] >= e["start"][i])


@pytest.mark.parametrize("maker", [
    lambda: wl.uniform_cube(6000, seed=3),
    lambda: wl.evrard(6000, seed=4),
    lambda: wl.plummer(6000, seed=5),
    lambda: wl.jittered_slab(20, 15, 10, seed=6),
])
def test_tree_invariants(oracle, maker):
    s = maker()
    t = oracle.OracleTree(s.x, s.y, s.z, bucket_size=8)
    _check_tree_invariants(t.export(), s.n, 8)


def test_coincident_particles_make_oversized_leaves(oracle):
    # all particles at one point: the root box is a point -> one oversized leaf
    x = np.full(100, 0.25, np.float32)
    t = oracle.OracleTree(x, x, x, bucket_size=16)
    e = t.export()
    assert t.num_nodes == 1 and e["oversized"][0] == 1 and e["count"][0] == 100
    # a coincident cluster inside a normal box recurses to depth 32, then stops
    rng = np.random.default_rng(7)
    p = rng.random((3, 200)).astype(np.float32)
    p[:, :50] = np.float32(0.3)
    t = oracle.OracleTree(p[0], p[1], p[2], bucket_size=16)
    e = t.export()
    assert t.max_depth == 32 and t.num_oversized == 1
    big = np.nonzero(e["oversized"])[0]
    assert e["depth"][big[0]] == 32 and e["count"][big[0]] == 50
    _check_tree_invariants(e, 200, 16)


def test_empty_and_single(oracle):
    t = oracle.OracleTree(np.zeros(0, np.float32), np.zeros(0, np.float32),
                          np.zeros(0, np.float32), bucket_size=4)
    nb, cnt = t.find(np.zeros(0, np.float32), 8)
    assert nb.shape == (0, 8)
    one = np.array([0.5], np.float32)
    t = oracle.OracleTree(one, one, one, bucket_size=4)
    nb, cnt = t.find(one, 4)
    assert cnt[0] == 0 and np.all(nb == -1)


# --------------------------------------------------------------- predicate / lists
def _lattice_truth(nx, ny, nz, h2_int=9):
    """Exact neighbour lists of the unjittered unit lattice with 2h = 3:
    all lattice offsets v != 0 with |v|^2 < 9, by integer enumeration."""
    offs = [v for v in itertools.product(range(-3, 4), repeat=3)
            if 0 < v[0] ** 2 + v[1] ** 2 + v[2] ** 2 < h2_int]
    out = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                lst = []
                for dx, dy, dz in offs:
                    a, b, c = i + dx, j + dy, k + dz
                    if 0 <= a < nx and 0 <= b < ny and 0 <= c < nz:
                        lst.append(a + nx * (b + ny * c))
                out.append(sorted(lst))
    return offs, out


def test_lattice_closed_form_counts_and_lists(oracle):
    nx, ny, nz = 9, 8, 7
    s = wl.lattice(nx, ny, nz, h=1.5)
    offs, truth = _lattice_truth(nx, ny, nz)
    # 93 lattice points with |v|^2 < 9 including the centre; the 30 points with
    # |v| = 3 exactly (D = R) are excluded by the strict predicate.
    assert len(offs) == 92
    assert sum(1 for v in itertools.product(range(-3, 4), repeat=3)
               if v[0] ** 2 + v[1] ** 2 + v[2] ** 2 == 9) == 30
    ngmax = 128
    for nb, cnt in (oracle.find_brute(s.x, s.y, s.z, s.h, ngmax),
                    oracle.OracleTree(s.x, s.y, s.z, bucket_size=16).find(s.h, ngmax)):
        for i in range(s.n):
            assert cnt[i] == len(truth[i])
            assert list(nb[i, :cnt[i]]) == truth[i]
            assert np.all(nb[i, cnt[i]:] == -1)
        # interior particles (>= 3 from every face) have exactly 92
        i = 4 + nx * (4 + ny * 3)
        assert cnt[i] == 92


def test_tiny_hand_checked_pairs(oracle):
    # D(0,1) = 1 = R(0) at h = 0.5: excluded (strict <)
    x = np.array([0, 1, 0], np.float32)
    y = np.array([0, 0, 2], np.float32)
    z = np.zeros(3, np.float32)
    nb, cnt = oracle.find_brute(x, y, z, np.full(3, 0.5, np.float32), 4)
    assert list(cnt) == [0, 0, 0]
    # asymmetric smoothing lengths: 0 sees 2 (D=4 < 4.84) but 2 does not see 0
    h = np.array([1.1, 0.6, 0.6], np.float32)
    nb, cnt = oracle.find_brute(x, y, z, h, 4)
    assert list(nb[0, :cnt[0]]) == [1, 2]
    assert list(nb[1, :cnt[1]]) == [0]
    assert list(nb[2, :cnt[2]]) == []
    # distance is summed in the stated order from float inputs
    assert oracle.distance2((0, 0, 0), (3, 4, 12)) == 169.0
    assert oracle.radius2(1.5) == 9.0


def test_coincident_neighbours_are_included_self_is_not(oracle):
    x = np.array([0.5, 0.5, 0.5, 0.9], np.float32)
    h = np.full(4, 0.1, np.float32)
    nb, cnt = oracle.find_brute(x, x, x, h, 4)
    assert list(nb[0, :cnt[0]]) == [1, 2]
    assert cnt[3] == 0


def test_pair_symmetry_uniform_h(oracle):
    s = wl.uniform_cube(3000, seed=11, target=60)
    nb, cnt = oracle.find_brute(s.x, s.y, s.z, s.h, 256)
    pairs = {(i, int(j)) for i in range(s.n) for j in nb[i, :cnt[i]]}
    assert all((j, i) in pairs for (i, j) in pairs)


def test_uniform_mean_count_matches_sphere_volume(oracle):
    s = wl.uniform_cube(20000, seed=12, target=100)
    t = oracle.OracleTree(s.x, s.y, s.z, bucket_size=16)
    _, cnt = t.find(s.h, 512)
    p = s.positions()
    r = 2 * float(s.h[0])
    inner = np.all((p > r) & (p < 1 - r), axis=1)
    expect = (s.n - 1) * 4.0 / 3.0 * math.pi * r ** 3
    got = cnt[inner].mean()
    assert abs(got - expect) < 4 * math.sqrt(expect / inner.sum()) + 0.5


def test_ngmax_keeps_smallest_indices(oracle):
    s = wl.uniform_cube(2000, seed=13, target=80)
    full, cfull = oracle.find_brute(s.x, s.y, s.z, s.h, 400)
    capped, ccap = oracle.find_brute(s.x, s.y, s.z, s.h, 16)
    assert np.array_equal(cfull, ccap)
    for i in range(s.n):
        k = min(16, cfull[i])
        assert np.array_equal(capped[i, :k], full[i, :k])


@pytest.mark.parametrize("maker,s_bucket", [
    (lambda: wl.uniform_cube(4000, seed=21), 16),
    (lambda: wl.evrard(4000, seed=22), 16),
    (lambda: wl.plummer(4000, seed=23, target=60), 8),
    (lambda: wl.jittered_slab(16, 16, 12, seed=24), 16),
    (lambda: wl.uniform_cube(3000, seed=25), 1),
])
def test_tree_walk_equals_brute_force(oracle, maker, s_bucket):
    s = maker()
    t = oracle.OracleTree(s.x, s.y, s.z, bucket_size=s_bucket)
    a, ca = t.find(s.h, 512)
    b, cb = oracle.find_brute(s.x, s.y, s.z, s.h, 512)
    assert np.array_equal(ca, cb)
    assert np.array_equal(a, b)


def test_tree_walk_equals_brute_force_degenerate(oracle):
    rng = np.random.default_rng(31)
    p = rng.random((3, 600)).astype(np.float32)
    p[:, :80] = np.float32(0.3)          # coincident cluster
    p[0, 80:120] = np.float32(0.5)       # particles on a plane
    p[:, 120] = 1.0                      # exactly at the upper box bound
    h = (rng.random(600) * 0.08 + 0.01).astype(np.float32)
    t = oracle.OracleTree(p[0], p[1], p[2], bucket_size=4)
    a, ca = t.find(h, 256)
    b, cb = oracle.find_brute(p[0], p[1], p[2], h, 256)
    assert np.array_equal(ca, cb) and np.array_equal(a, b)


# --------------------------------------------------------------- M4 density
def test_m4_normalisation_and_continuity(oracle):
    from scipy.integrate import quad
    for h in (0.3, 1.0, 1.5):
        val, err = quad(lambda r: 4 * math.pi * r * r * oracle.kernel_w(r, h), 0, 2 * h,
                        points=[h], limit=200)
        assert abs(val - 1.0) < 1e-10
        assert oracle.kernel_w(0.0, h) == pytest.approx(1.0 / (math.pi * h ** 3), rel=1e-15)
        assert oracle.kernel_w(2 * h, h) == 0.0
    eps = 1e-7
    for q in (1.0, 2.0):
        lo, hi = oracle.m4_shape(q - eps), oracle.m4_shape(q + eps)
        assert abs(lo - hi) < 1e-6
        dlo = (oracle.m4_shape(q - eps) - oracle.m4_shape(q - 2 * eps)) / eps
        dhi = (oracle.m4_shape(q + 2 * eps) - oracle.m4_shape(q + eps)) / eps
        assert abs(dlo - dhi) < 1e-5
    assert oracle.m4_shape(1.0) == 0.25


def test_density_gather_form(oracle):
    # isolated particle: self term only
    x = np.array([0.0, 10.0], np.float32)
    z = np.zeros(2, np.float32)
    h = np.array([0.5, 0.7], np.float32)
    m = np.array([2.0, 3.0], np.float32)
    t = oracle.OracleTree(x, z, z, bucket_size=1)
    rho = t.density(h, m)
    assert rho[0] == pytest.approx(2.0 / (math.pi * 0.125), rel=1e-15)
    # pair at distance 0.6 with different h: particle 0 (2h=1.0) sees 1 and uses
    # its own h and the neighbour's mass; particle 1 (h=0.2, 2h=0.4) does not
    x = np.array([0.0, 0.6], np.float32)
    h = np.array([0.5, 0.2], np.float32)
    t = oracle.OracleTree(x, z, z, bucket_size=1)
    rho = t.density(h, m)
    d = float(np.float32(0.6))
    assert rho[0] == pytest.approx(2.0 * oracle.kernel_w(0, 0.5) + 3.0 * oracle.kernel_w(d, 0.5), rel=1e-14)
    assert rho[1] == pytest.approx(3.0 * oracle.kernel_w(0, float(np.float32(0.2))), rel=1e-14)


def test_density_lattice_is_riemann_sum_of_unit_integral(oracle):
    s = wl.lattice(11, 11, 11, h=1.5)
    t = oracle.OracleTree(s.x, s.y, s.z, bucket_size=16)
    rho = t.density(s.h, s.m)
    i = 5 + 11 * (5 + 11 * 5)
    # sum_v W(|v|, h) over the unit lattice approximates the integral of W = 1
    assert abs(rho[i] * s.n - 1.0) < 0.01


# --------------------------------------------------------------- octree mode
def test_octree_mode_is_the_perfect_octree_on_a_power_of_two_lattice(oracle):
    # 8x8x8 unit lattice, box [0,7]^3, s = 1: every split halves at the cell
    # middle, 4 lattice points per side -> depth 3, 1 + 8 + 64 internal cells,
    # every leaf one particle
    s = wl.lattice(8, 8, 8, h=0.5)
    t = oracle.OracleTree(s.x, s.y, s.z, bucket_size=1, octree=True)
    e = t.export()
    internal = e["b"] > 0
    assert np.all(e["b"][internal] == 2)
    assert internal.sum() == 73 and t.max_depth == 3
    leaf = ~internal
    assert np.all(e["count"][leaf] == 1)
    # the b-tree of the same lattice is one level (b0 = 8)
    tb = oracle.OracleTree(s.x, s.y, s.z, bucket_size=1)
    assert tb.export()["b"][0] == 8 and tb.max_depth == 1


def test_octree_and_btree_give_the_same_lists(oracle):
    s = wl.evrard(5000, seed=91, target=60)
    a = oracle.OracleTree(s.x, s.y, s.z, bucket_size=8, octree=True).find(s.h, 256)
    b = oracle.OracleTree(s.x, s.y, s.z, bucket_size=8).find(s.h, 256)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    _check_tree_invariants(oracle.OracleTree(s.x, s.y, s.z, bucket_size=8, octree=True).export(),
                           s.n, 8)


# --------------------------------------------------------------- k = 2 trees
@pytest.mark.parametrize("s_", [1, 3, 4, 16])
def test_branching_factor_k2_closed_form(oracle, s_):
    for n in list(range(s_ + 1, 400)) + [10**6, 10**6 + 1, 123457]:
        b = oracle.branching_factor(n, s_, k=2)
        assert b >= 2 and b * b * s_ >= n
        assert b == 2 or (b - 1) ** 2 * s_ < n
    assert oracle.branching_factor(100, 1, k=2) == 10
    assert oracle.branching_factor(101, 1, k=2) == 11


def _planar_lattice(nx, ny):
    i = np.arange(nx * ny)
    x, y = (i % nx).astype(np.float32), (i // nx).astype(np.float32)
    return x, y, np.zeros_like(x), np.full(x.size, 0.75, np.float32)


def test_k2_perfect_quadtree_on_a_planar_lattice(oracle):
    # 8x8 lattice, box [0,7]^2, s = 1, b forced to 2: every split halves x
    # and y at the middle -> depth 3, 1 + 4 + 16 internal cells, 64 leaves of one
    x, y, z, h = _planar_lattice(8, 8)
    t = oracle.OracleTree(x, y, z, bucket_size=1, octree=True, dim=2)
    e = t.export()
    internal = e["b"] > 0
    assert internal.sum() == 21 and t.max_depth == 3
    assert np.all(e["count"][~internal] <= 1)
    assert e["count"][~internal].sum() == 64 and np.sum(e["count"][~internal] == 1) == 64
    _check_tree_invariants(e, 64, 1, k=2)
    # the b-tree: b0 = 8 (8^2 * 1 >= 64), one level of 64 single-particle cells
    tb = oracle.OracleTree(x, y, z, bucket_size=1, dim=2)
    eb = tb.export()
    assert eb["b"][0] == 8 and tb.max_depth == 1 and (eb["b"] > 0).sum() == 1


def test_k2_tree_never_splits_z_and_lists_are_the_definition(oracle):
    s = wl.uniform_cube(4000, seed=31, target=40)
    t = oracle.OracleTree(s.x, s.y, s.z, bucket_size=8, dim=2)
    e = t.export()
    _check_tree_invariants(e, s.n, 8, k=2)
    assert np.all(e["lo"][:, 2] == e["lo"][0, 2]) and np.all(e["hi"][:, 2] == e["hi"][0, 2])
    nb, cnt = t.find(s.h, 128)
    rnb, rcnt = oracle.find_brute(s.x, s.y, s.z, s.h, 128)
    assert np.array_equal(cnt, rcnt) and np.array_equal(nb, rnb)
    # a planar set: the 2-D lists
    x, y, z, h = _planar_lattice(30, 20)
    t2 = oracle.OracleTree(x, y, z, bucket_size=4, dim=2)
    nb2, cnt2 = t2.find(h, 32)
    rnb2, rcnt2 = oracle.find_brute(x, y, z, h, 32)
    assert np.array_equal(cnt2, rcnt2) and np.array_equal(nb2, rnb2)
    # interior points of the unit lattice with h = 0.75: |v|^2 < 2.25 gives
    # the 8 points at distance 1 and sqrt(2)
    interior = (x >= 2) & (x <= 27) & (y >= 2) & (y <= 17)
    assert np.all(cnt2[interior] == 8)

