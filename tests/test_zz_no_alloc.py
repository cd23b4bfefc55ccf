"""The allocation-free fused search (btree_find_neighbors_density_noalloc).

It exists for callers that cannot allocate device memory at the moment they
search -- a loop that forbids allocation after set-up, or a host framework
that owns all device memory -- and keeps its one scratch buffer in a fixed
array inside the library.  Called through the C ABI, it must give what the
regular entry point gives, also on the second of two calls in a row (the
array keeps the previous call's contents).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bt():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1910_02639_gb300 as m
    return m


def _run(bt, s, ngmax, noalloc):
    import torch
    dev = torch.device("cuda:0")
    x, y, z, h, m = (torch.from_numpy(np.ascontiguousarray(a)).to(dev)
                     for a in (s.x, s.y, s.z, s.h, s.m))
    tree = bt.btree_build(x, y, z, h, bucket_size=16)
    nb = torch.full((s.n * ngmax,), -1, dtype=torch.int32, device=dev)
    cnt = torch.empty(s.n, dtype=torch.int32, device=dev)
    rho = torch.empty(s.n, dtype=torch.float32, device=dev)
    if noalloc:
        bt.btree_find_neighbors_density_noalloc(tree, m, ngmax, nb, cnt, rho)
    else:
        bt.btree_find_neighbors_density(tree, m, ngmax, nb, cnt, rho)
    torch.cuda.synchronize()
    out = (nb.cpu().numpy(), cnt.cpu().numpy(), rho.cpu().numpy())
    tree.free()
    return out


def test_noalloc_matches_regular_on_two_calls_in_a_row(bt):
    from paper_1910_02639_gb300 import workloads as wl
    sets = [wl.evrard(200_000, seed=81), wl.uniform_cube(30_000, seed=82, target=80)]
    for s in sets:  # the second call reuses the array the first one filled
        ref_nb, ref_cnt, ref_rho = _run(bt, s, 256, noalloc=False)
        nb, cnt, rho = _run(bt, s, 256, noalloc=True)
        assert np.array_equal(cnt, ref_cnt)
        assert np.array_equal(nb, ref_nb)
        # the same kernel on the same inputs: the densities agree bit for bit
        assert np.array_equal(rho.view(np.int32), ref_rho.view(np.int32))


def test_noalloc_rejects_trees_above_its_limit(bt):
    import torch
    from paper_1910_02639_gb300 import workloads as wl
    limit = bt.btree_noalloc_max_particles()
    assert limit == 1 << 21
    s = wl.uniform_cube(limit + 1, seed=83, target=40)
    dev = torch.device("cuda:0")
    x, y, z, h, m = (torch.from_numpy(a).to(dev) for a in (s.x, s.y, s.z, s.h, s.m))
    tree = bt.btree_build(x, y, z, h, bucket_size=16)
    nb = torch.empty(1 * s.n, dtype=torch.int32, device=dev)
    cnt = torch.empty(s.n, dtype=torch.int32, device=dev)
    rho = torch.empty(s.n, dtype=torch.float32, device=dev)
    with pytest.raises(bt.BtreeError) as ei:
        bt.btree_find_neighbors_density_noalloc(tree, m, 1, nb, cnt, rho)
    assert ei.value.status == bt.BT_ERR_CAPACITY
    tree.free()
