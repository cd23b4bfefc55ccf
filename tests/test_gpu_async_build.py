"""Asynchronous rebuilds.  The first build of a handle runs synchronously (it
sets the buffer capacities, growing them if needed); a rebuild of the same
sets with the same parameters (new positions) is one CUDA-graph launch with
device-driven level and ratio loops, and the call returns without waiting
for the device.  Its host-side summary is read by the next call that needs
it; its device-detected conditions by btree_status."""
import time

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


def _dev(s):
    import torch
    return [torch.from_numpy(a).to("cuda:0") for a in (s.x, s.y, s.z, s.h, s.m)]


def _rows(bt, tree, m, n, g=128):
    import torch
    nb = torch.full((n * g,), -1, dtype=torch.int32, device="cuda:0")
    cnt = torch.empty(n, dtype=torch.int32, device="cuda:0")
    rho = torch.empty(n, dtype=torch.float32, device="cuda:0")
    bt.btree_find_neighbors_density(tree, m, g, nb, cnt, rho)
    return nb, cnt, rho


def test_rebuild_returns_before_the_device_finishes(bt):
    import torch
    s = wl.uniform_cube(1_000_000, seed=95, target=60)
    x, y, z, h, m = _dev(s)
    tree = bt.btree_build(x, y, z, h, bucket_size=16)  # synchronous: sets capacities
    torch.cuda.synchronize()
    # new positions, same sets and parameters: queued behind a 0.3 s kernel
    s2 = wl.uniform_cube(1_000_000, seed=96, target=60)
    x2, y2, z2, h2, m2 = _dev(s2)
    torch.cuda.synchronize()
    torch.cuda._sleep(int(0.3 * 2.0e9))  # a bounded clock spin on the current stream
    t0 = time.perf_counter()
    bt.btree_build(x2, y2, z2, h2, bucket_size=16, tree=tree)
    dt = time.perf_counter() - t0
    nb, cnt, rho = _rows(bt, tree, m2, s2.n)  # queued after the build, no host wait either
    ev = torch.cuda.Event()
    ev.record()
    busy = not ev.query()
    torch.cuda.synchronize()
    assert busy, "the device had already finished: the calls waited for it"
    assert dt < 0.1, f"btree_build took {dt:.3f} s of host time"
    # the results are those of a fresh synchronous build of the new positions
    ref = bt.btree_build(x2, y2, z2, h2, bucket_size=16)
    rnb, rcnt, rrho = _rows(bt, ref, m2, s2.n)
    torch.cuda.synchronize()
    assert torch.equal(cnt, rcnt) and torch.equal(nb, rnb)
    assert torch.equal(rho.view(torch.int32), rrho.view(torch.int32))
    assert bt.btree_get_info(tree)["num_groups"] == bt.btree_get_info(ref)["num_groups"]
    tree.free()
    ref.free()


def test_async_rebuild_reports_through_status(bt):
    import torch
    rng = np.random.default_rng(97)
    p = rng.random((3, 20_000)).astype(np.float32)
    p[:, :50] = np.float32(0.25)  # 50 coincident particles: an oversized leaf
    h = np.full(20_000, 0.01, np.float32)
    s = wl._pack(p[0], p[1], p[2], h)
    x, y, z, hh, m = _dev(s)
    tree = bt.btree_build(x, y, z, hh, bucket_size=16)
    assert tree.status == bt.BT_WARN_OVERSIZED_LEAF  # synchronous first build
    bt.btree_status(tree)  # clears the device status word
    bt.btree_build(x, y, z, hh, bucket_size=16, tree=tree)  # asynchronous rebuild
    nb, cnt, _ = _rows(bt, tree, m, s.n)
    assert bt.btree_status(tree) == bt.BT_WARN_OVERSIZED_LEAF
    info = bt.btree_get_info(tree)
    assert info["num_oversized"] >= 1
    torch.cuda.synchronize()
    tree.free()
