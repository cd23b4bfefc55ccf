"""Batched BuildTree: many independent, uneven particle sets in one build
(btree_build_batched), searched and summed by the same find / density calls.

Each set's tree must be the oracle's tree of that set alone (Algorithm 1 with
the set's own s, alpha, beta, or the octree of Sec. 2), and its neighbour
lists, counts and densities must be identical -- bit for bit, densities
included -- to those of the same set built and searched alone.
"""
import numpy as np
import pytest

from paper_1910_02639_gb300 import workloads as wl
from tests._gpu import compare_trees, run_gpu

pytestmark = pytest.mark.gpu

NGMAX = 256


@pytest.fixture(scope="module")
def bt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1910_02639_gb300 as m
    return m


def _concat(sets):
    off = np.zeros(len(sets) + 1, np.int64)
    off[1:] = np.cumsum([s.n for s in sets])
    cat = lambda k: np.concatenate([getattr(s, k) for s in sets]).astype(np.float32)
    return off, cat("x"), cat("y"), cat("z"), cat("h"), cat("m")


def run_batched(bt, sets, params=None, ngmax=NGMAX):
    import torch
    dev = torch.device("cuda:0")
    off, *arrs = _concat(sets)
    x, y, z, h, m = (torch.from_numpy(a).to(dev) for a in arrs)
    n = int(off[-1])
    tree = bt.btree_build_batched(x, y, z, h, off, params)
    nb = torch.full((max(n, 1) * ngmax,), -1, dtype=torch.int32, device=dev)
    cnt = torch.full((max(n, 1),), -7, dtype=torch.int32, device=dev)
    rho = torch.empty(max(n, 1), dtype=torch.float32, device=dev)
    bt.btree_find_neighbors_density(tree, m, ngmax, nb, cnt, rho)
    torch.cuda.synchronize()
    nbh = nb.view(-1, ngmax)[:n].cpu().numpy()
    cnth, rhoh = cnt[:n].cpu().numpy(), rho[:n].cpu().numpy()
    out = [dict(nb=nbh[off[i]:off[i + 1]], cnt=cnth[off[i]:off[i + 1]],
                rho=rhoh[off[i]:off[i + 1]]) for i in range(len(sets))]
    return tree, off, out


def _coincident(n):
    return wl._pack(np.full(n, 0.25), np.full(n, -1.0), np.full(n, 3.0), np.full(n, 0.1),
                    name="coincident")


def _mixed_sets():
    """Every path of the builder in one batch: empty set, one particle, a set
    that is one leaf (n = s), the warp builder (<= 256), big cells, clustered
    and flat sets, coincident particles."""
    return [
        wl.evrard(40_000, seed=501, target=60),
        wl._pack(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0)),
        wl.uniform_cube(1, seed=502),
        wl.uniform_cube(16, seed=503, target=10),
        wl.uniform_cube(17, seed=504, target=10),
        wl.plummer(200, seed=505, target=40),
        wl.uniform_cube(257, seed=506, target=50),
        _coincident(40),
        wl.plummer(30_000, seed=507, target=80),
        wl.jittered_slab(40, 25, 1, jitter=0.1, h=1.5, seed=508),
        wl.uniform_cube(9_000, seed=509, target=120),
        wl.sphere_1r(3_000, seed=510, target=100),
    ]


def _assert_same(a, b, what):
    assert np.array_equal(a["cnt"], b["cnt"]), what + ": counts"
    assert np.array_equal(a["nb"], b["nb"]), what + ": lists"
    assert np.array_equal(a["rho"].view(np.int32), b["rho"].view(np.int32)), what + ": densities"


def test_batched_equals_each_set_alone(bt):
    sets = _mixed_sets()
    tree, off, res = run_batched(bt, sets)
    info = bt.btree_get_info(tree)
    assert info["n"] == off[-1]
    tree.free()
    for i, s in enumerate(sets):
        if s.n == 0:
            continue
        alone = run_gpu(s, bucket_size=16, ngmax=NGMAX, density=True)
        alone["tree"].free()
        _assert_same(res[i], alone, "set %d (%s, n=%d)" % (i, s.name, s.n))


def test_empty_sets_at_both_ends_and_chunk_boundaries(bt):
    """Empty sets first, last and in a row; sets whose sizes straddle the
    4096-particle blocks of the root passes (bounding box, one-leaf sets)."""
    empty = wl._pack(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0))
    sets = [empty, empty, wl.uniform_cube(4096, seed=521, target=40), empty,
            wl.uniform_cube(4097, seed=522, target=40), wl.uniform_cube(12, seed=523, target=8),
            wl.evrard(8191, seed=524, target=50), empty, empty]
    tree, off, res = run_batched(bt, sets)
    tree.free()
    for i, s in enumerate(sets):
        if s.n == 0:
            continue
        alone = run_gpu(s, bucket_size=16, ngmax=NGMAX, density=True)
        alone["tree"].free()
        _assert_same(res[i], alone, "set %d (n=%d)" % (i, s.n))


def test_thousands_of_tiny_sets(bt, oracle):
    """2000 sets of 0 to 40 particles (many empty, many one leaf, some split
    by the warp builder) in one batch: every list, count and density against
    the oracle's brute force on that set."""
    rng = np.random.default_rng(77)
    sets = []
    for i in range(2000):
        n = int(rng.integers(0, 41))
        sets.append(wl.uniform_cube(n, seed=1000 + i, target=8) if n else
                    wl._pack(np.zeros(0), np.zeros(0), np.zeros(0), np.zeros(0)))
    params = [dict(bucket_size=int(rng.choice([1, 4, 16]))) for _ in sets]
    tree, off, res = run_batched(bt, sets, params=params, ngmax=64)
    tree.free()
    worst = 0.0
    for i, s in enumerate(sets):
        if s.n == 0:
            continue
        ref_nb, ref_cnt = oracle.find_brute(s.x, s.y, s.z, s.h, 64)
        assert np.array_equal(res[i]["cnt"], ref_cnt), f"set {i}: counts"
        assert np.array_equal(res[i]["nb"], ref_nb), f"set {i}: lists"
        ref_rho = oracle.OracleTree(s.x, s.y, s.z, bucket_size=16).density(s.h, s.m)
        worst = max(worst, float(np.max(np.abs(res[i]["rho"] - ref_rho) / ref_rho)))
    assert worst < 1e-5


def test_batched_trees_match_the_oracle_per_set(bt, oracle):
    sets = _mixed_sets()
    params = [dict(bucket_size=(16, 5, 1, 8)[i % 4], beta=(0.5, 0.0, 1.0)[i % 3],
                   octree=(i % 5 == 2)) for i in range(len(sets))]
    tree, off, res = run_batched(bt, sets, params)
    e = bt.btree_export(tree)
    tree.free()
    for i, (s, p) in enumerate(zip(sets, params)):
        ot = oracle.OracleTree(s.x, s.y, s.z, bucket_size=p["bucket_size"], beta=p["beta"],
                               octree=p["octree"])
        compare_trees(e, ot.export(), s.n, root=i, off=int(off[i]))
        ref_nb, ref_cnt = oracle.find_brute(s.x, s.y, s.z, s.h, NGMAX)
        assert np.array_equal(res[i]["cnt"], ref_cnt), "set %d counts" % i
        used = np.arange(NGMAX)[None, :] < np.minimum(ref_cnt, NGMAX)[:, None]
        assert np.array_equal(np.where(used, ref_nb, -1), res[i]["nb"]), "set %d lists" % i


def test_octree_sets_give_the_btree_lists(bt):
    sets = [wl.evrard(50_000, seed=511, target=80), wl.plummer(20_000, seed=512, target=60)]
    _, _, bres = run_batched(bt, sets, dict(bucket_size=16))
    _, _, ores = run_batched(bt, sets, dict(bucket_size=16, octree=True))
    for i in range(len(sets)):
        assert np.array_equal(bres[i]["cnt"], ores[i]["cnt"])
        assert np.array_equal(bres[i]["nb"], ores[i]["nb"])


def test_many_uneven_sets_density_matches_oracle(bt, oracle):
    # 48 sets, log-uniform sizes 100 .. 30000, the kinds of the batched workload
    sets = wl.batched_sets(48, seed=513, nmin=100, nmax=30_000)
    _, off, res = run_batched(bt, sets)
    for i, s in enumerate(sets):
        ot = oracle.OracleTree(s.x, s.y, s.z, bucket_size=16)
        nb, cnt = ot.find(s.h, NGMAX)
        assert np.array_equal(res[i]["cnt"], cnt), "set %d counts" % i
        rho = ot.density(s.h, s.m)
        rel = np.abs(res[i]["rho"].astype(np.float64) - rho) / rho
        assert rel.max() < 1e-5, "set %d density" % i


def test_batched_order_of_sets_does_not_matter(bt):
    sets = wl.batched_sets(12, seed=514, nmin=50, nmax=20_000)
    _, _, a = run_batched(bt, sets)
    perm = np.random.default_rng(5).permutation(len(sets))
    _, _, b = run_batched(bt, [sets[k] for k in perm])
    for j, k in enumerate(perm):
        _assert_same(a[k], b[j], "set %d" % k)


def test_batched_argument_errors(bt):
    import torch
    x = torch.zeros(10, device="cuda:0")
    with pytest.raises(ValueError):
        bt.btree_build_batched(x, x, x, x, [0, 5, 9])
    with pytest.raises(bt.BtreeError) as ei:
        bt.btree_build_batched(x, x, x, x, [0, 6, 5, 10])
    assert ei.value.status == bt.BT_ERR_ARG
    with pytest.raises(bt.BtreeError):
        bt.btree_build_batched(x, x, x, x, [0, 10], dict(bucket_size=0))


@pytest.mark.parametrize("params", [
    dict(group_size=8), dict(group_size=16), dict(group_size=1),
    dict(bucket_size=64, beta=0.25, group_size=16), dict(bucket_size=8, beta=0.75),
    dict(find_compact=True), dict(find_compact=True, bucket_size=8, group_size=16),
    dict(pack_leaves=True), dict(pack_leaves=True, bucket_size=8, beta=0.25, find_compact=True),
    dict(pack_leaves=True, bucket_size=4, group_size=16),
    [dict(find_compact=bool(i % 2), bucket_size=(8, 16, 32)[i % 3]) for i in range(10)],
])
def test_tuning_knobs_never_change_results(bt, params):
    # s, beta and the work-unit size change the tree and the schedule only:
    # lists, counts and densities must stay bit-identical
    sets = wl.batched_sets(10, seed=515, nmin=300, nmax=40_000)
    _, _, ref = run_batched(bt, sets)
    _, _, got = run_batched(bt, sets, params)
    for i in range(len(sets)):
        _assert_same(got[i], ref[i], "set %d with %s" % (i, params))


def test_plain_path_helper_matches_batched(bt):
    import torch
    from paper_1910_02639_gb300.batch import DeviceSets, list_checksum
    sets = wl.batched_sets(8, seed=516, nmin=500, nmax=20_000)
    ds = DeviceSets(sets, "cuda:0", NGMAX)
    ds.run_plain()
    torch.cuda.synchronize()
    ref = [ds.results(i) for i in range(len(sets))]
    c_ref = list_checksum(ds.nb, ds.cnt, NGMAX)
    ds.run_batched()
    torch.cuda.synchronize()
    for i in range(len(sets)):
        nb, cnt, rho = ds.results(i)
        k = np.minimum(cnt, NGMAX)
        used = np.arange(NGMAX)[None, :] < k[:, None]
        assert np.array_equal(cnt, ref[i][1])
        assert np.array_equal(np.where(used, nb, -1), np.where(used, ref[i][0], -1))
        assert np.array_equal(rho.view(np.int32), ref[i][2].view(np.int32))
    assert list_checksum(ds.nb, ds.cnt, NGMAX) == c_ref
    ds.free()


def test_autotuner_table_and_params(bt):
    from paper_1910_02639_gb300.autotune import Tuner, set_class
    sets = wl.batched_sets(6, seed=517, nmin=2_000, nmax=50_000)
    tu = Tuner("cuda:0", NGMAX, reps=1, sample_particles=100_000)
    table = tu.tune(sets)
    assert set(table) == {set_class(s) for s in sets}
    for e in table.values():
        assert e["bucket_size"] in (8, 16, 32, 64) and e["beta"] in (0.25, 0.5, 0.75)
        assert e["group_size"] in (16, 32) and e["find_compact"] in (False, True) and e["ms"] > 0
    params = tu.params_for(sets)
    _, _, ref = run_batched(bt, sets)
    _, _, got = run_batched(bt, sets, params)
    for i in range(len(sets)):
        _assert_same(got[i], ref[i], "set %d tuned" % i)


# ------------------------------------------------------------------ graph form
def run_graph(bt, sets, params=None, ngmax=NGMAX, tree=None, density=True, bufs=None):
    import torch
    dev = torch.device("cuda:0")
    off, *arrs = _concat(sets)
    n = int(off[-1])
    if bufs is None:
        x, y, z, h, m = (torch.from_numpy(a).to(dev) for a in arrs)
        nb = torch.full((max(n, 1) * ngmax,), -1, dtype=torch.int32, device=dev)
        cnt = torch.full((max(n, 1),), -7, dtype=torch.int32, device=dev)
        rho = torch.empty(max(n, 1), dtype=torch.float32, device=dev)
    else:
        x, y, z, h, m, nb, cnt, rho = bufs
        for d, a in zip((x, y, z, h, m), arrs):
            d.copy_(torch.from_numpy(a))
        nb.fill_(-1)
    tree = bt.btree_build_find_batched(x, y, z, h, off, ngmax, nb, cnt,
                                       m=m if density else None, rho=rho if density else None,
                                       params=params, tree=tree)
    torch.cuda.synchronize()
    nbh = nb.view(-1, ngmax)[:n].cpu().numpy()
    cnth, rhoh = cnt[:n].cpu().numpy(), rho[:n].cpu().numpy()
    out = [dict(nb=nbh[off[i]:off[i + 1]], cnt=cnth[off[i]:off[i + 1]],
                rho=rhoh[off[i]:off[i + 1]]) for i in range(len(sets))]
    return tree, off, out, (x, y, z, h, m, nb, cnt, rho)


def test_graph_form_equals_separate_calls(bt):
    sets = _mixed_sets()
    t0, _, ref = run_batched(bt, sets)
    t0.free()
    t1, _, got, _ = run_graph(bt, sets)
    info = bt.btree_get_info(t1)
    assert info["num_groups"] > 0 and info["max_depth"] >= 2
    t1.free()
    for i in range(len(sets)):
        _assert_same(got[i], ref[i], "set %d graph" % i)


def test_graph_relaunch_with_new_parameters_and_new_inputs(bt):
    sets = wl.batched_sets(9, seed=519, nmin=300, nmax=40_000)
    _, _, ref = run_batched(bt, sets)
    tree, off, got, bufs = run_graph(bt, sets)
    for i in range(len(sets)):
        _assert_same(got[i], ref[i], "first launch, set %d" % i)
    # same buffers and sizes: the captured graph is relaunched; per-set
    # parameters are read on the device at each launch
    for params in (dict(bucket_size=8, beta=0.25), dict(bucket_size=64, group_size=16),
                   dict(find_compact=True), None):
        tree, _, got, bufs = run_graph(bt, sets, params=params, tree=tree, bufs=bufs)
        for i in range(len(sets)):
            _assert_same(got[i], ref[i], "relaunch %s, set %d" % (params, i))
    # other inputs of another size through the same handle: a new capture
    sets2 = wl.batched_sets(5, seed=520, nmin=1000, nmax=80_000)
    _, _, ref2 = run_batched(bt, sets2)
    tree, _, got2, _ = run_graph(bt, sets2, tree=tree)
    for i in range(len(sets2)):
        _assert_same(got2[i], ref2[i], "recapture, set %d" % i)
    tree.free()


def test_graph_form_without_density_and_plummer_tails(bt, oracle):
    sets = [wl.plummer(3000, seed=521, target=120), wl.plummer(20_000, seed=522, target=90),
            wl.uniform_cube(5000, seed=523, target=70)]
    tree, _, got, _ = run_graph(bt, sets, density=False, ngmax=512)
    tree.free()
    for i, s in enumerate(sets):
        ref_nb, ref_cnt = oracle.OracleTree(s.x, s.y, s.z, bucket_size=16).find(s.h, 512)
        assert np.array_equal(got[i]["cnt"], ref_cnt), "set %d counts" % i
        used = np.arange(512)[None, :] < np.minimum(ref_cnt, 512)[:, None]
        assert np.array_equal(np.where(used, ref_nb, -1), got[i]["nb"]), "set %d lists" % i


def test_graph_form_rejects_nonfinite_and_recovers(bt):
    bad = wl.uniform_cube(3000, seed=524, target=50)
    bad.x[17] = np.nan
    good = wl.uniform_cube(3000, seed=525, target=50)
    with pytest.raises(bt.BtreeError) as ei:
        run_graph(bt, [good, bad])
    assert ei.value.status == bt.BT_ERR_NONFINITE
    _, _, ref = run_batched(bt, [good])
    tree, _, got, _ = run_graph(bt, [good])
    _assert_same(got[0], ref[0], "after a rejected input")
    tree.free()


def test_graph_form_counts_its_kernels(bt):
    sets = wl.batched_sets(6, seed=526, nmin=2000, nmax=60_000)
    l0 = bt.btree_kernel_launches()
    tree, _, _, _ = run_graph(bt, sets)
    l1 = bt.btree_kernel_launches()
    tree.free()
    assert 20 <= l1 - l0 <= 400


# ------------------------------------------------------------------ compressed rows
def test_csr_rows_are_the_full_lists(bt, oracle):
    import torch
    sets = [wl.uniform_cube(6000, seed=527, target=400), wl.plummer(5000, seed=528, target=90)]
    dev = torch.device("cuda:0")
    off, *arrs = _concat(sets)
    x, y, z, h, m = (torch.from_numpy(a).to(dev) for a in arrs)
    n = int(off[-1])
    tree = bt.btree_build_batched(x, y, z, h, off, [dict(), dict(find_compact=True)])
    offsets = torch.empty(n + 1, dtype=torch.int64, device=dev)
    rho = torch.empty(n, dtype=torch.float32, device=dev)
    total = bt.btree_find_neighbors_csr(tree, offsets, m=m, rho=rho)  # sizes only
    nbrs = torch.full((total + 5,), -3, dtype=torch.int32, device=dev)
    assert bt.btree_find_neighbors_csr(tree, offsets, nbrs) == total
    with pytest.raises(bt.BtreeError) as ei:
        bt.btree_find_neighbors_csr(tree, offsets, nbrs[:total - 1])
    assert ei.value.status == bt.BT_ERR_CAPACITY
    torch.cuda.synchronize()
    o = offsets.cpu().numpy()
    rows = nbrs.cpu().numpy()
    assert o[0] == 0 and o[-1] == total and np.all(rows[total:] == -3)
    # fused fixed-row density is the same bits
    _, _, ref = run_batched(bt, sets, [dict(), dict(find_compact=True)], ngmax=2048)
    rho_h = rho.cpu().numpy()
    for i, s in enumerate(sets):
        a = int(off[i])
        cnt = np.diff(o[a:a + s.n + 1])
        ref_nb, ref_cnt = oracle.find_brute(s.x, s.y, s.z, s.h, s.n)  # full rows
        assert np.array_equal(cnt, ref_cnt), "set %d counts" % i
        for r in range(s.n):
            assert np.array_equal(rows[o[a + r]:o[a + r + 1]], ref_nb[r, :ref_cnt[r]]), "set %d row %d" % (i, r)
        assert np.array_equal(rho_h[a:a + s.n].view(np.int32), ref[i]["rho"].view(np.int32))
    tree.free()


# ------------------------------------------------------------------ k = 2
def _planar(n, seed, target):
    rng = np.random.default_rng(seed)
    x, y = rng.random((2, n)).astype(np.float32)
    # 2-D number density n per unit area: h from pi (2h)^2 n = target
    h = np.full(n, np.sqrt(target / (np.pi * n)) / 2, np.float32)
    return wl._pack(x, y, np.zeros(n, np.float32), h, name="planar")


def test_k2_sets_trees_and_lists(bt, oracle):
    sets = [_planar(20_000, 530, 40), _planar(3_000, 531, 25), wl.uniform_cube(8_000, seed=532, target=60),
            wl.plummer(4_000, seed=533, target=50), _planar(17, 534, 5)]
    params = [dict(dim=2), dict(dim=2, octree=True), dict(dim=2, bucket_size=8),
              dict(dim=2, find_compact=True), dict(dim=2)]
    tree, off, res = run_batched(bt, sets, params, ngmax=512)
    e = bt.btree_export(tree)
    tree.free()
    for i, (s, p) in enumerate(zip(sets, params)):
        ot = oracle.OracleTree(s.x, s.y, s.z, bucket_size=p.get("bucket_size", 16),
                               octree=p.get("octree", False), dim=2)
        compare_trees(e, ot.export(), s.n, root=i, off=int(off[i]), k=2)
        ref_nb, ref_cnt = oracle.find_brute(s.x, s.y, s.z, s.h, 512)
        assert np.array_equal(res[i]["cnt"], ref_cnt), "set %d counts" % i
        used = np.arange(512)[None, :] < np.minimum(ref_cnt, 512)[:, None]
        assert np.array_equal(np.where(used, ref_nb, -1), res[i]["nb"]), "set %d lists" % i
        rho = ot.density(s.h, s.m)
        assert (np.abs(res[i]["rho"] - rho) / rho).max() < 1e-5, "set %d density" % i
    # the 2-D trees give the same lists and densities as the 3-D trees
    _, _, res3 = run_batched(bt, sets, None, ngmax=512)
    for i in range(len(sets)):
        _assert_same(res[i], res3[i], "set %d k=2 vs k=3" % i)


def test_pack_rows_equals_csr_rows(bt):
    import torch
    sets = [wl.uniform_cube(20_000, seed=535, target=80), wl.sphere_1r(15_000, seed=536, target=120),
            wl.uniform_cube(3_000, seed=537, target=60)]
    g = 1024
    tree, off, res = run_batched(bt, sets, ngmax=g)
    dev = torch.device("cuda:0")
    n = int(off[-1])
    assert max(int(r["cnt"].max()) for r in res) <= g
    # fixed rows again on the device, then packed
    rows = torch.full((n * g,), -1, dtype=torch.int32, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev)
    bt.btree_find_neighbors(tree, g, rows, cnt)
    offs_p = torch.empty(n + 1, dtype=torch.int64, device=dev)
    total = bt.btree_pack_rows(tree, rows, cnt, g, offs_p)
    csr_p = torch.full((total,), -9, dtype=torch.int32, device=dev)
    assert bt.btree_pack_rows(tree, rows, cnt, g, offs_p, csr_p) == total
    offs_c = torch.empty(n + 1, dtype=torch.int64, device=dev)
    csr_c = torch.empty(total, dtype=torch.int32, device=dev)
    assert bt.btree_find_neighbors_csr(tree, offs_c, csr_c) == total
    assert torch.equal(offs_p, offs_c) and torch.equal(csr_p, csr_c)
    # capped rows pack only their first ngmax entries
    small = 8
    rows8 = torch.empty(n * small, dtype=torch.int32, device=dev)
    bt.btree_find_neighbors(tree, small, rows8, cnt)
    t8 = bt.btree_pack_rows(tree, rows8, cnt, small, offs_p)
    assert t8 == int(cnt.clamp(max=small).to(torch.int64).sum())
    tree.free()


def test_half_rows_are_the_upper_half_of_the_full_rows(bt):
    import torch
    # uniform h: the relation is symmetric, every pair once; variable h: still
    # exactly {j in N(i) : j > i}
    sets = [wl.jittered_slab(30, 20, 12, jitter=0.1, h=1.5, seed=538), wl.evrard(8_000, seed=539, target=60),
            wl.plummer(3_000, seed=540, target=80)]
    dev = torch.device("cuda:0")
    off, *arrs = _concat(sets)
    x, y, z, h, m = (torch.from_numpy(a).to(dev) for a in arrs)
    n = int(off[-1])
    tree = bt.btree_build_batched(x, y, z, h, off, [dict(), dict(find_compact=True), dict(bucket_size=8)])
    of = torch.empty(n + 1, dtype=torch.int64, device=dev)
    tot = bt.btree_find_neighbors_csr(tree, of)
    full = torch.empty(tot, dtype=torch.int32, device=dev)
    bt.btree_find_neighbors_csr(tree, of, full)
    oh = torch.empty(n + 1, dtype=torch.int64, device=dev)
    toth = bt.btree_find_neighbors_csr(tree, oh, half=True)
    halfr = torch.empty(toth, dtype=torch.int32, device=dev)
    bt.btree_find_neighbors_csr(tree, oh, halfr, half=True)
    with pytest.raises(bt.BtreeError):
        bt.btree_find_neighbors_csr(tree, oh, m=m, rho=torch.empty_like(m), half=True)
    torch.cuda.synchronize()
    of, full, oh, halfr = of.cpu().numpy(), full.cpu().numpy(), oh.cpu().numpy(), halfr.cpu().numpy()
    for i in range(n):
        s_ = np.searchsorted(off, i, side="right") - 1
        local = i - off[s_]
        row = full[of[i]:of[i + 1]]
        assert np.array_equal(halfr[oh[i]:oh[i + 1]], row[row > local]), "row %d" % i
    a, b = int(off[0]), int(off[1])
    assert 2 * (oh[b] - oh[a]) == of[b] - of[a]  # the slab (uniform h): each pair once
    tree.free()
