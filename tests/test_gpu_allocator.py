"""The allocator hook of btree_build (bt_allocator, include/btree.h), driven
through the C ABI from Python callbacks.

A production caller routes the tree's buffers through its own device memory
manager; here that is PyTorch's caching allocator.  Host-side fault
injection: an allocator that refuses its k-th request must make the build
return BT_ERR_OOM, leave the handle freeable (every buffer it did hand out
comes back), and the next build with a working allocator must succeed.
No GPU fault is involved: the failure is a NULL returned on the host.
"""
import numpy as np
import pytest

from paper_1910_02639_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1910_02639_gb300 as m
    return m


class Counting:
    """PyTorch's caching allocator, counted; refuses request number `fail_at`."""

    def __init__(self, bt, fail_at=None):
        import torch
        self.live = {}
        self.allocs = self.frees = self.refused = 0
        self.fail_at = fail_at
        dev = torch.device("cuda", torch.cuda.current_device())

        def alloc(n, stream):
            self.allocs += 1
            if self.fail_at is not None and self.allocs == self.fail_at:
                self.refused += 1
                return 0
            p = torch.cuda.caching_allocator_alloc(n, dev, stream)
            self.live[p] = n
            return p

        def free(p, stream):
            self.frees += 1
            assert self.live.pop(p, None) is not None, "freed a pointer it did not hand out"
            torch.cuda.caching_allocator_delete(p)

        self.allocator = bt.Allocator(alloc, free)


def _search(bt, tree, s, ngmax=128):
    import torch
    dev = torch.device("cuda:0")
    m = torch.from_numpy(s.m).to(dev)
    nb = torch.full((s.n * ngmax,), -1, dtype=torch.int32, device=dev)
    cnt = torch.empty(s.n, dtype=torch.int32, device=dev)
    rho = torch.empty(s.n, dtype=torch.float32, device=dev)
    bt.btree_find_neighbors_density(tree, m, ngmax, nb, cnt, rho)
    torch.cuda.synchronize()
    return nb.cpu().numpy(), cnt.cpu().numpy(), rho.cpu().numpy()


def _dev(s):
    import torch
    dev = torch.device("cuda:0")
    return [torch.from_numpy(a).to(dev) for a in (s.x, s.y, s.z, s.h)]


def test_torch_caching_allocator_owns_the_tree(bt):
    s = wl.evrard(50_000, seed=91)
    x, y, z, h = _dev(s)
    ref_tree = bt.btree_build(x, y, z, h, bucket_size=16)
    ref = _search(bt, ref_tree, s)
    ref_tree.free()
    c = Counting(bt)
    tree = bt.btree_build(x, y, z, h, bucket_size=16, allocator=c.allocator)
    got = _search(bt, tree, s)  # the fused search allocates its mass buffer through the hook too
    assert c.allocs > 10 and len(c.live) == c.allocs - c.frees
    for a, b in zip(got, ref):
        assert np.array_equal(a.view(np.int32), b.view(np.int32))
    tree.free()
    assert c.frees == c.allocs and not c.live, "every buffer returned through the hook"


@pytest.mark.parametrize("fail_at", [1, 3, 12])
def test_refused_allocation_gives_oom_and_recovers(bt, fail_at):
    s = wl.uniform_cube(20_000, seed=92, target=60)
    x, y, z, h = _dev(s)
    c = Counting(bt, fail_at=fail_at)
    tree = bt.Tree()
    with pytest.raises(bt.BtreeError) as ei:
        bt.btree_build(x, y, z, h, bucket_size=16, tree=tree, allocator=c.allocator)
    assert ei.value.status == bt.BT_ERR_OOM
    assert c.refused == 1
    tree.free()  # the handle is still valid: everything it holds comes back
    assert c.frees == c.allocs - c.refused and not c.live
    # the next build (a fresh handle, a working allocator) succeeds
    ok = Counting(bt)
    t2 = bt.btree_build(x, y, z, h, bucket_size=16, allocator=ok.allocator)
    nb, cnt, _ = _search(bt, t2, s)
    ref_tree = bt.btree_build(x, y, z, h, bucket_size=16)
    rnb, rcnt, _ = _search(bt, ref_tree, s)
    assert np.array_equal(cnt, rcnt) and np.array_equal(nb, rnb)
    t2.free()
    ref_tree.free()
    assert ok.frees == ok.allocs and not ok.live


def test_oom_mid_rebuild_keeps_the_handle_usable(bt):
    # a tree built once, then rebuilt in place with an allocator that refuses
    # a later request: OOM, then a rebuild with a working allocator into the
    # same handle gives the right lists
    s = wl.plummer(15_000, seed=93)
    x, y, z, h = _dev(s)
    c = Counting(bt)
    tree = bt.btree_build(x, y, z, h, bucket_size=16, allocator=c.allocator)
    bad = Counting(bt, fail_at=4)
    with pytest.raises(bt.BtreeError) as ei:
        bt.btree_build(x, y, z, h, bucket_size=8, tree=tree, allocator=bad.allocator)
    assert ei.value.status == bt.BT_ERR_OOM
    good = Counting(bt)
    bt.btree_build(x, y, z, h, bucket_size=16, tree=tree, allocator=good.allocator)
    nb, cnt, _ = _search(bt, tree, s)
    ref_tree = bt.btree_build(x, y, z, h, bucket_size=16)
    rnb, rcnt, _ = _search(bt, ref_tree, s)
    assert np.array_equal(cnt, rcnt) and np.array_equal(nb, rnb)
    tree.free()
    ref_tree.free()
    assert good.frees == good.allocs and not good.live
