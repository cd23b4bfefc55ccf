"""One particle set split over ranks (slabs along x + one halo exchange):
the union of the ranks' rows, counts and densities equals a single run over
the whole set.  CPU: gloo ranks with the oracle as the per-rank search.
GPU: two gloo ranks sharing the one GPU (their kernels never wait on each
other; the exchange is on the host), against a single GPU run, bit for bit."""
import os
import socket

import numpy as np
import pytest

from paper_1910_02639_gb300 import workloads as wl


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _mixed_set():
    """A uniform cube next to a Plummer sphere with its very wide outskirts
    (some h reach across the whole set, so halos are large)."""
    a = wl.uniform_cube(2500, seed=21, target=60)
    b = wl.plummer(1500, seed=22, target=40)
    cat = lambda k, sh=0.0: np.concatenate([getattr(a, k), getattr(b, k) + sh]).astype(np.float32)
    return dict(x=cat("x", 1.5), y=cat("y"), z=cat("z"), h=cat("h"), m=cat("m"))


def _oracle_compute(x, y, z, h, m, ngmax, bucket_size, density):
    import torch
    import oracle
    xs, ys, zs, hs, ms = (t.cpu().numpy() for t in (x, y, z, h, m))
    nb, cnt = oracle.find_brute(xs, ys, zs, hs, ngmax)
    rho = None
    if density:
        rho = torch.from_numpy(oracle.OracleTree(xs, ys, zs, bucket_size=bucket_size).density(hs, ms))
    return torch.from_numpy(nb), torch.from_numpy(cnt), rho


def _rank_main(rank, world, port, data, ngmax, use_gpu, q):
    import torch
    import torch.distributed as dist
    from paper_1910_02639_gb300.halo import decomposed_find
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = data["x"].shape[0]
    mine = np.arange(rank, n, world)  # any initial distribution will do
    dev = torch.device("cuda:0") if use_gpu else torch.device("cpu")
    t = lambda k: torch.from_numpy(data[k][mine]).to(dev)
    out = decomposed_find(t("x"), t("y"), t("z"), t("h"), t("m"), torch.from_numpy(mine),
                          ngmax, compute=None if use_gpu else _oracle_compute)
    q.put((rank, out["gidx"].numpy(), out["nb"].numpy(), out["cnt"].numpy(),
           out["rho"].numpy(), out["halo"]))
    dist.destroy_process_group()


def _run_ranks(world, data, ngmax, use_gpu):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, data, ngmax, use_gpu, q))
          for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in ps:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in ps)
    res.sort()
    g = np.concatenate([r[1] for r in res])
    o = np.argsort(g)
    return (g[o], np.concatenate([r[2] for r in res])[o], np.concatenate([r[3] for r in res])[o],
            np.concatenate([r[4] for r in res])[o], [r[5] for r in res])


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_equal_the_whole_set(world):
    import oracle
    data = _mixed_set()
    n = data["x"].shape[0]
    ngmax = 64
    g, nb, cnt, rho, halos = _run_ranks(world, data, ngmax, use_gpu=False)
    assert np.array_equal(g, np.arange(n))  # every particle owned by exactly one rank
    ref_nb, ref_cnt = oracle.find_brute(data["x"], data["y"], data["z"], data["h"], ngmax)
    assert np.array_equal(cnt, ref_cnt)
    assert np.array_equal(nb, ref_nb)
    ref_rho = oracle.OracleTree(data["x"], data["y"], data["z"]).density(data["h"], data["m"])
    assert np.max(np.abs(rho - ref_rho) / ref_rho) < 1e-12
    assert all(hc > 0 for hc in halos)


def test_slab_cuts_and_halo_width_on_a_lattice():
    """Lattice slab, 2 ranks: the halo each rank receives is exactly the
    lattice planes within 2h (1 + 2^-20) of its own particles."""
    s = wl.jittered_slab(40, 10, 10, jitter=0.0, h=1.5, seed=1)
    data = dict(x=s.x, y=s.y, z=s.z, h=s.h, m=s.m)
    g, nb, cnt, rho, halos = _run_ranks(2, data, 128, use_gpu=False)
    # cut at x = 20, own extents [0, 19] and [20, 39], R = 3(1 + 2^-20): rank 0
    # receives the planes x = 20..22, rank 1 the planes x = 17..19 (100 each)
    assert halos == [300, 300]
    assert np.array_equal(g, np.arange(s.n))


@pytest.mark.gpu
def test_two_ranks_on_one_gpu_equal_a_single_run():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from tests import _gpu
    s = wl.evrard(40000, seed=31)
    data = dict(x=s.x, y=s.y, z=s.z, h=s.h, m=s.m)
    ngmax = 256
    r = _gpu.run_gpu(s, bucket_size=16, ngmax=ngmax, density=True)
    g, nb, cnt, rho, halos = _run_ranks(2, data, ngmax, use_gpu=True)
    assert np.array_equal(g, np.arange(s.n))
    assert np.array_equal(cnt, r["cnt"])
    full = np.minimum(cnt, ngmax)
    mask = np.arange(ngmax)[None, :] < full[:, None]
    assert np.array_equal(np.where(mask, nb, -1), np.where(mask, r["nb"], -1))
    assert np.array_equal(rho.view(np.int32), r["rho"].view(np.int32))
