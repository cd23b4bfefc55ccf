"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Lists and counts must be bit-identical; the FP32 density must be within
1e-5 relative of the FP64 oracle for rows that are not truncated."""
import itertools
import math

import numpy as np
import pytest

from paper_1910_02639_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

DENS_TOL = 1e-5


@pytest.fixture(scope="module")
def bt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1910_02639_gb300 as m
    return m


@pytest.fixture(scope="module")
def gpu(bt):
    from tests import _gpu
    return _gpu


def _brute(oracle, s, ngmax):
    return oracle.find_brute(s.x, s.y, s.z, s.h, ngmax)


def _assert_lists(r, ref_nb, ref_cnt):
    assert np.array_equal(r["cnt"], ref_cnt), \
        f"counts differ at {np.nonzero(r['cnt'] != ref_cnt)[0][:10]}"
    bad = np.nonzero(np.any(r["nb"] != ref_nb, axis=1))[0]
    assert bad.size == 0, f"rows differ at {bad[:10]}"


# ------------------------------------------------------------------ plain small config
def test_uniform_32768_full_brute_force(bt, gpu, oracle):
    """Plain small case: 32768 uniform particles, ~100 neighbours, s=16,
    ngmax=256; every row against the O(n^2) definition."""
    s = wl.uniform_cube(32768, seed=1911)
    r = gpu.run_gpu(s, bucket_size=16, ngmax=256, density=True)
    ref_nb, ref_cnt = _brute(oracle, s, 256)
    _assert_lists(r, ref_nb, ref_cnt)
    assert 80 < ref_cnt.mean() < 105
    ot = oracle.OracleTree(s.x, s.y, s.z, bucket_size=16)
    ref_rho = ot.density(s.h, s.m)
    rel = np.abs(r["rho"] - ref_rho) / ref_rho
    assert rel.max() < DENS_TOL
    info = bt.btree_get_info(r["tree"])
    assert info["root_b"] == 13


@pytest.mark.parametrize("case", ["uniform", "evrard", "plummer", "slab", "clustered"])
def test_tree_shape_matches_oracle(bt, gpu, oracle, case):
    makers = {
        "uniform": lambda: wl.uniform_cube(20000, seed=41),
        "evrard": lambda: wl.evrard(60000, seed=42),
        "plummer": lambda: wl.plummer(30000, seed=43),
        "slab": lambda: wl.jittered_slab(40, 30, 20, seed=44),
        "clustered": lambda: _clustered(5000, 45),
    }
    s = makers[case]()
    for bucket in (16, 5):
        r = gpu.run_gpu(s, bucket_size=bucket, ngmax=8)
        e = bt.btree_export(r["tree"])
        ot = oracle.OracleTree(s.x, s.y, s.z, bucket_size=bucket)
        gpu.compare_trees(e, ot.export(), s.n)
        info = bt.btree_get_info(r["tree"])
        assert info["max_depth"] == ot.max_depth
        # every particle exactly once in tree order
        assert np.array_equal(np.sort(e["order"]), np.arange(s.n))


def _clustered(n, seed):
    rng = np.random.default_rng(seed)
    p = rng.random((3, n)).astype(np.float32)
    p[:, : n // 2] = (rng.random((3, n // 2)) * 0.001 + 0.3).astype(np.float32)
    p[:, n // 2: n // 2 + 40] = np.float32(0.7)  # coincident -> oversized leaf at depth 32
    h = (rng.random(n) * 0.02 + 0.001).astype(np.float32)
    return wl._pack(p[0], p[1], p[2], h, name="clustered")


def test_near_pairs_grow_the_tree_buffers(bt, gpu, oracle):
    """Pairs of nearly coincident particles at s = 1: each pair is a chain of
    two-particle cells down to the level where its particles part (about 15
    levels below the root, Algorithm 1 with b = 2), so the tree holds far
    more internal nodes and sub-cells than the build's first estimate of its
    buffers (3n/(s+1) nodes, 16n/s sub-cells).  The build grows them, builds
    again, and gives the oracle's tree and the brute-force lists."""
    rng = np.random.default_rng(61)
    npair = 1500
    a = (rng.random((3, npair)) * 0.9 + 0.05).astype(np.float32)
    d = ((rng.random((3, npair)) - 0.5) * 2e-6).astype(np.float32)
    p = np.concatenate([a, a + d], axis=1)
    h = np.full(2 * npair, 0.02, np.float32)
    s = wl._pack(p[0], p[1], p[2], h, name="near_pairs")
    n = s.n
    r = gpu.run_gpu(s, bucket_size=1, ngmax=64)
    info = bt.btree_get_info(r["tree"])
    assert info["num_nodes"] > 3 * n // 2 + 1024 + 1, "the first node estimate sufficed: no growth exercised"
    assert info["num_slots"] > 16 * n + 4096
    ot = oracle.OracleTree(s.x, s.y, s.z, bucket_size=1)
    gpu.compare_trees(bt.btree_export(r["tree"]), ot.export(), n)
    assert info["max_depth"] == ot.max_depth
    ref_nb, ref_cnt = _brute(oracle, s, 64)
    _assert_lists(r, ref_nb, ref_cnt)
    # a rebuild in place (same sets, new positions: the asynchronous form)
    # keeps the grown buffers and gives the same result for the same input
    r2 = gpu.run_gpu(s, bucket_size=1, ngmax=64, tree=r["tree"])
    _assert_lists(r2, ref_nb, ref_cnt)
    assert bt.btree_get_info(r2["tree"])["num_nodes"] == info["num_nodes"]
    r["tree"].free()


@pytest.mark.parametrize("case", ["evrard", "plummer", "slab", "clustered"])
def test_lists_match_brute_force_varied(bt, gpu, oracle, case):
    makers = {
        "evrard": lambda: wl.evrard(20000, seed=51),
        "plummer": lambda: wl.plummer(20000, seed=52, target=80),
        "slab": lambda: wl.jittered_slab(30, 25, 20, seed=53),
        "clustered": lambda: _clustered(8000, 54),
    }
    s = makers[case]()
    r = gpu.run_gpu(s, bucket_size=16, ngmax=512)
    ref_nb, ref_cnt = _brute(oracle, s, 512)
    _assert_lists(r, ref_nb, ref_cnt)


def test_lattice_closed_form(bt, gpu, oracle):
    """Unjittered lattice with h = 1.5: interior particles have exactly 92
    neighbours (strict <: the 30 lattice points at distance 3 are out)."""
    s = wl.lattice(24, 20, 16, h=1.5)
    r = gpu.run_gpu(s, bucket_size=16, ngmax=128, density=True)
    ref_nb, ref_cnt = _brute(oracle, s, 128)
    _assert_lists(r, ref_nb, ref_cnt)
    i = 10 + 24 * (10 + 20 * 8)
    assert r["cnt"][i] == 92


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("n", [0, 1, 2, 16, 17, 33, 255, 256, 257, 4097])
def test_sizes_and_ragged_tails(bt, gpu, oracle, n):
    s = wl.uniform_cube(max(n, 1), seed=60 + n, target=30)
    if n == 0:
        s = wl._pack(*(np.zeros(0, np.float32),) * 4)
    r = gpu.run_gpu(s, bucket_size=16, ngmax=64)
    if n:
        ref_nb, ref_cnt = _brute(oracle, s, 64)
        _assert_lists(r, ref_nb, ref_cnt)


def test_all_coincident(bt, gpu, oracle):
    x = np.full(3000, 0.25, np.float32)
    s = wl._pack(x, x, x, np.full(3000, 0.1, np.float32))
    r = gpu.run_gpu(s, bucket_size=16, ngmax=64)
    assert np.all(r["cnt"] == 2999)
    assert np.array_equal(r["nb"][5], np.r_[0:5, 6:65].astype(np.int32))
    assert r["tree"].status == bt.BT_WARN_OVERSIZED_LEAF
    assert bt.btree_status(r["tree"]) == bt.BT_WARN_NGMAX


def test_degenerate_geometry(bt, gpu, oracle):
    rng = np.random.default_rng(61)
    p = rng.random((3, 3000)).astype(np.float32)
    p[:, :300] = np.float32(0.3)        # coincident cluster
    p[0, 300:700] = np.float32(0.5)     # a plane
    p[:, 700] = 1.0                     # on the upper box bound
    p[2, :] = np.where(np.arange(3000) % 7 == 0, np.float32(0.0), p[2])
    h = (rng.random(3000) * 0.05 + 0.005).astype(np.float32)
    h[5] = 0.0
    s = wl._pack(p[0], p[1], p[2], h)
    r = gpu.run_gpu(s, bucket_size=8, ngmax=400)
    ref_nb, ref_cnt = _brute(oracle, s, 400)
    _assert_lists(r, ref_nb, ref_cnt)
    e = bt.btree_export(r["tree"])
    ot = oracle.OracleTree(s.x, s.y, s.z, bucket_size=8)
    gpu.compare_trees(e, ot.export(), s.n)


def test_flat_slab_zero_width_dimension(bt, gpu, oracle):
    rng = np.random.default_rng(62)
    x = rng.random(5000).astype(np.float32)
    y = rng.random(5000).astype(np.float32)
    z = np.zeros(5000, np.float32)
    s = wl._pack(x, y, z, np.full(5000, 0.02, np.float32))
    r = gpu.run_gpu(s, bucket_size=16, ngmax=128)
    ref_nb, ref_cnt = _brute(oracle, s, 128)
    _assert_lists(r, ref_nb, ref_cnt)


def test_large_h_windowed_path(bt, gpu, oracle):
    """Candidate sets larger than one window (1024) go through the windowed
    path: same lists, capped rows keep the smallest indices."""
    s = wl.uniform_cube(6000, seed=63, target=2500)
    r = gpu.run_gpu(s, bucket_size=16, ngmax=300, density=True)
    ref_nb, ref_cnt = _brute(oracle, s, 300)
    _assert_lists(r, ref_nb, ref_cnt)
    assert ref_cnt.max() > 1024
    assert bt.btree_status(r["tree"]) == bt.BT_WARN_NGMAX
    ot = oracle.OracleTree(s.x, s.y, s.z, bucket_size=16)
    ref_rho = ot.density(s.h, s.m)
    rel = np.abs(r["rho"] - ref_rho) / ref_rho
    assert rel.max() < DENS_TOL


def test_windowed_path_on_a_large_set(bt, gpu, oracle):
    """Work units whose candidates span several windows but only a small part
    of a large set take the windowed path (not the scan)."""
    s = wl.uniform_cube(150_000, seed=66, target=1500)
    r = gpu.run_gpu(s, bucket_size=16, ngmax=300, density=True)
    ot = oracle.OracleTree(s.x, s.y, s.z, bucket_size=16)
    ref_nb, ref_cnt = ot.find(s.h, 300)
    _assert_lists(r, ref_nb, ref_cnt)
    assert ref_cnt.max() > 1024
    rel = np.abs(r["rho"] - ot.density(s.h, s.m)) / ot.density(s.h, s.m)
    assert rel.max() < DENS_TOL


def test_huge_h_scan_mode(bt, gpu, oracle):
    """A few particles whose 2h covers most of the set (the outskirts of a
    Plummer sphere with analytic h): their work units scan the set in index
    order.  Lists, counts and densities as the definition."""
    base = wl.uniform_cube(20_000, seed=67, target=60)
    h = base.h.copy()
    rng = np.random.default_rng(67)
    far = rng.choice(base.n, 200, replace=False)
    h[far] = rng.uniform(0.2, 0.9, far.size).astype(np.float32)
    # and one tight cluster of large-h particles, so whole work units are wide
    x, y, z = base.x.copy(), base.y.copy(), base.z.copy()
    x[:64], y[:64], z[:64] = 0.9 + 1e-3 * rng.random((3, 64)).astype(np.float32)
    h[:64] = 0.45
    s = wl._pack(x, y, z, h)
    r = gpu.run_gpu(s, bucket_size=16, ngmax=512, density=True)
    ref_nb, ref_cnt = _brute(oracle, s, 512)
    _assert_lists(r, ref_nb, ref_cnt)
    assert ref_cnt.max() > 5000
    ot = oracle.OracleTree(s.x, s.y, s.z, bucket_size=16)
    rel = np.abs(r["rho"] - ot.density(s.h, s.m)) / ot.density(s.h, s.m)
    assert rel.max() < DENS_TOL


def test_boundary_pairs_exact_predicate(bt, gpu, oracle):
    """Pairs placed at D = R within a few ulps: the FP32 filter must defer to
    the binary64 predicate."""
    rng = np.random.default_rng(64)
    n = 4000
    base = rng.random((n, 3)).astype(np.float32) * np.float32(10.0)
    h = np.full(n, 0.25, np.float32)
    # partner of every even particle at distance exactly 2h along a random axis,
    # nudged by -2..2 ulps
    for i in range(0, n - 1, 2):
        ax = i % 3
        q = base[i].copy()
        v = np.float32(base[i, ax] + np.float32(0.5))
        v = np.nextafter(v, np.float32(np.inf) if (i // 2) % 2 else np.float32(-np.inf))
        for _ in range((i // 4) % 3):
            v = np.nextafter(v, np.float32(np.inf))
        q[ax] = v
        base[i + 1] = q
    s = wl._pack(base[:, 0], base[:, 1], base[:, 2], h)
    r = gpu.run_gpu(s, bucket_size=8, ngmax=64)
    ref_nb, ref_cnt = _brute(oracle, s, 64)
    _assert_lists(r, ref_nb, ref_cnt)


def test_ngmax_one_and_capping(bt, gpu, oracle):
    s = wl.uniform_cube(5000, seed=65, target=50)
    for ngmax in (1, 7):
        r = gpu.run_gpu(s, bucket_size=16, ngmax=ngmax)
        ref_nb, ref_cnt = _brute(oracle, s, ngmax)
        _assert_lists(r, ref_nb, ref_cnt)


@pytest.mark.parametrize("bucket,beta", [(1, 0.5), (8, 0.0), (8, 1.0), (64, 0.5), (300, 0.5)])
def test_parameters_change_tree_not_lists(bt, gpu, oracle, bucket, beta):
    s = wl.evrard(12000, seed=66, target=60)
    r = gpu.run_gpu(s, bucket_size=bucket, beta=beta, ngmax=256)
    ref_nb, ref_cnt = _brute(oracle, s, 256)
    _assert_lists(r, ref_nb, ref_cnt)
    e = bt.btree_export(r["tree"])
    ot = oracle.OracleTree(s.x, s.y, s.z, bucket_size=bucket, beta=beta)
    gpu.compare_trees(e, ot.export(), s.n)


def test_nonfinite_rejected(bt, gpu):
    s = wl.uniform_cube(1000, seed=67)
    s.x[10] = np.nan
    with pytest.raises(bt.BtreeError) as ei:
        gpu.run_gpu(s)
    assert ei.value.status == -5


def test_rebuild_in_place_and_determinism(bt, gpu):
    s = wl.evrard(50000, seed=68)
    r1 = gpu.run_gpu(s, ngmax=256, density=True)
    r2 = gpu.run_gpu(s, ngmax=256, density=True, tree=r1["tree"])
    assert np.array_equal(r1["nb"], r2["nb"]) and np.array_equal(r1["cnt"], r2["cnt"])
    assert np.array_equal(r1["rho"].view(np.int32), r2["rho"].view(np.int32))
    s2 = wl.uniform_cube(3000, seed=69)
    r3 = gpu.run_gpu(s2, ngmax=128, tree=r1["tree"])  # smaller set into the same handle
    assert r3["cnt"].shape == (3000,)


def test_standalone_density_consumer(bt, gpu, oracle):
    import torch
    s = wl.plummer(15000, seed=70, target=70)
    r = gpu.run_gpu(s, ngmax=512, density=True)
    m = torch.from_numpy(s.m).cuda()
    rho2 = torch.empty(s.n, dtype=torch.float32, device="cuda")
    bt.sph_density(r["tree"], m, r["nb_dev"], r["cnt_dev"], 512, rho2)
    torch.cuda.synchronize()
    ot = oracle.OracleTree(s.x, s.y, s.z, bucket_size=16)
    ref = ot.density(s.h, s.m)
    full = r["cnt"] <= 512
    for got in (r["rho"], rho2.cpu().numpy()):
        rel = np.abs(got[full] - ref[full]) / ref[full]
        assert rel.max() < DENS_TOL


# ------------------------------------------------------------------ full-size configs
@pytest.mark.slow
def test_evrard_1e6_full_rows(bt, gpu, oracle):
    """Evrard-like collapse, 1e6 particles, ngmax 512: every row, count and
    density against the oracle tree walk (itself pinned to brute force)."""
    s = wl.evrard(1_000_000, seed=1912)
    r = gpu.run_gpu(s, bucket_size=16, ngmax=512, density=True)
    ot = oracle.OracleTree(s.x, s.y, s.z, bucket_size=16)
    step = 125_000
    for q0 in range(0, s.n, step):
        ref_nb, ref_cnt = ot.find(s.h, 512, q0, q0 + step)
        assert np.array_equal(r["cnt"][q0:q0 + step], ref_cnt)
        assert np.array_equal(r["nb"][q0:q0 + step], ref_nb)
    e = bt.btree_export(r["tree"])
    gpu.compare_trees(e, ot.export(), s.n)
    ref_rho = ot.density(s.h, s.m)
    rel = np.abs(r["rho"].astype(np.float64) - ref_rho) / ref_rho
    assert rel.max() < DENS_TOL, f"density error {rel.max():.3g} at {int(rel.argmax())}"


def _jittered_lattice_mean_count(jitter, radius, samples=400_000, seed=3):
    """Monte Carlo expectation of the neighbour count of an interior particle
    of a unit lattice with uniform per-coordinate jitter."""
    rng = np.random.default_rng(seed)
    d = (rng.uniform(-jitter, jitter, (samples, 3)) - rng.uniform(-jitter, jitter, (samples, 3)))
    lim = int(math.ceil(radius + 2 * jitter))
    total = 0.0
    for v in itertools.product(range(-lim, lim + 1), repeat=3):
        if v == (0, 0, 0):
            continue
        r0 = math.sqrt(v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
        if r0 + 2 * jitter * math.sqrt(3) < radius:
            total += 1.0
        elif r0 - 2 * jitter * math.sqrt(3) < radius:
            w = d + np.array(v, dtype=np.float64)
            total += float(np.mean((w * w).sum(axis=1) < radius * radius))
    return total


@pytest.mark.slow
def test_slab_1e7_every_row(bt, gpu, oracle):
    """Jittered slab, 1e7 particles, in the launch configuration the
    benchmark times (one-set batched build, compact shape): every row, count
    and density against the oracle tree walk; the plain btree_build path
    gives the same bits; pair symmetry (uniform h) on a sample; the interior
    mean count against its expectation."""
    import torch
    s = wl.jittered_slab()
    x, y, z, h, m = gpu.to_dev(s)
    tree = bt.btree_build_batched(x, y, z, h, np.array([0, s.n], np.int64),
                                  [dict(bucket_size=16, alpha=0.5, beta=0.5, find_compact=True)])
    nb = torch.full((s.n * 256,), -1, dtype=torch.int32, device=x.device)
    cnt = torch.empty(s.n, dtype=torch.int32, device=x.device)
    rho = torch.empty(s.n, dtype=torch.float32, device=x.device)
    bt.btree_find_neighbors_density(tree, m, 256, nb, cnt, rho)
    torch.cuda.synchronize()
    cnt_h, rho_h = cnt.cpu().numpy(), rho.cpu().numpy()
    ot = oracle.OracleTree(s.x, s.y, s.z, bucket_size=16)
    step = 1_000_000
    worst = 0.0
    for q0 in range(0, s.n, step):
        q1 = min(q0 + step, s.n)
        ref_nb, ref_cnt = ot.find(s.h, 256, q0, q1)
        assert np.array_equal(cnt_h[q0:q1], ref_cnt), f"counts differ in [{q0}, {q1})"
        got = nb[q0 * 256:q1 * 256].view(-1, 256).cpu().numpy()
        bad = np.nonzero(np.any(got != ref_nb, axis=1))[0]
        assert bad.size == 0, f"rows differ at {q0 + bad[:10]}"
        ref_rho = ot.density(s.h, s.m, q0, q1)
        worst = max(worst, float(np.max(np.abs(rho_h[q0:q1].astype(np.float64) - ref_rho) / ref_rho)))
    assert worst < DENS_TOL, f"density error {worst:.3g}"
    # the plain path (btree_build, default shape): the same bits
    r = gpu.run_gpu(s, bucket_size=16, ngmax=256, density=True)
    assert torch.equal(r["cnt_dev"], cnt)
    assert torch.equal(r["nb_dev"], nb)
    assert torch.equal(r["rho_dev"].view(torch.int32), rho.view(torch.int32))
    # symmetry: j in N(i) <=> i in N(j) for sampled i
    rows = r["nb"]
    rng = np.random.default_rng(1)
    for i in rng.choice(s.n, 500, replace=False):
        for j in rows[i, :cnt_h[i]]:
            assert i in rows[j, :cnt_h[j]]
    # interior mean count = sum over lattice offsets v != 0 of
    # P(|v + d_j - d_i| < 3), jitter differences triangular on [-0.2, 0.2]
    ix = np.arange(s.n)
    gx, gy, gz = ix % 400, (ix // 400) % 250, ix // 100000
    inner = (gx > 5) & (gx < 394) & (gy > 5) & (gy < 244) & (gz > 5) & (gz < 94)
    assert abs(cnt_h[inner].mean() - _jittered_lattice_mean_count(0.1, 3.0)) < 0.15
    tree.free()
    r["tree"].free()
    del r, nb, rows
    torch.cuda.empty_cache()


@pytest.mark.slow
def test_batched_256_sets_every_row(bt, oracle):
    """The 256-set workload at full size (35.6 M particles) as one CUDA-graph
    launch, every tuning knob in use across the sets: every row, count and
    density of every set against the oracle tree of that set."""
    import torch
    from paper_1910_02639_gb300.batch import DeviceSets
    sets = wl.batched_sets(256, seed=1914)
    knobs = [dict(), dict(find_compact=True), dict(bucket_size=8, pack_leaves=True),
             dict(bucket_size=64, beta=0.75, group_size=16), dict(bucket_size=32, beta=0.25)]
    params = [knobs[i % len(knobs)] for i in range(len(sets))]
    ds = DeviceSets(sets, "cuda:0", 256)
    ds.run_graph(params)
    torch.cuda.synchronize()
    cnt_all, rho_all = ds.cnt.cpu().numpy(), ds.rho.cpu().numpy()
    worst = 0.0
    for i, s in enumerate(sets):
        a = int(ds.offsets[i])
        p = {**dict(bucket_size=16, beta=0.5), **params[i]}
        ot = oracle.OracleTree(s.x, s.y, s.z, bucket_size=p["bucket_size"], beta=p["beta"])
        ref_nb, ref_cnt = ot.find(s.h, 256)
        assert np.array_equal(cnt_all[a:a + s.n], ref_cnt), f"set {i}: counts differ"
        got = ds.nb[a * 256:(a + s.n) * 256].view(-1, 256).cpu().numpy()
        k = np.minimum(ref_cnt, 256)
        written = np.arange(256)[None, :] < k[:, None]
        assert np.array_equal(got[written], ref_nb[written]), f"set {i}: rows differ"
        ref_rho = ot.density(s.h, s.m)
        worst = max(worst, float(np.max(np.abs(rho_all[a:a + s.n].astype(np.float64) - ref_rho) / ref_rho)))
        del ot, ref_nb, got
    assert worst < DENS_TOL, f"density error {worst:.3g}"
    ds.free()
    torch.cuda.empty_cache()


@pytest.mark.gpu
def test_arith_rates_measured():
    """The FMA-rate diagnostic runs and orders the rates as the FP32 filter
    assumes: binary64 far below FP32."""
    import paper_1910_02639_gb300 as bt
    r = bt.btree_arith_rates()
    assert r["fp32_gflops"] > 1e3 and r["fp32x2_gflops"] > 1e3 and r["fp64_gflops"] > 10
    assert r["fp64_gflops"] < 0.5 * r["fp32_gflops"]
