"""Serving loop: continuous batching of build + find + density requests.

Every request's neighbour rows, counts and densities must be bit-identical to
those of the same set run alone on the plain path, whatever batch it was
admitted in; admission must respect the HBM budget; batches on different
slots overlap."""
import numpy as np
import pytest

from paper_1910_02639_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
NGMAX = 128


@pytest.fixture(scope="module")
def srv_mod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1910_02639_gb300 import serving
    return serving


def _requests(serving, nreq, seed, nmin, nmax, spread=0.0):
    specs = wl.request_stream(nreq, seed=seed, nmin=nmin, nmax=nmax)
    return [serving.make_request(i, spread * i / max(nreq, 1), wl.make_set(k, n, s, t))
            for i, (_, k, n, s, t) in enumerate(specs)]


def _grab(store):
    def f(res):
        g = NGMAX
        cnt = res.cnt.cpu().numpy()
        nb = res.nb.view(-1, g).cpu().numpy()
        used = np.arange(g)[None, :] < np.minimum(cnt, g)[:, None]
        store[res.rid] = (cnt, np.where(used, nb, -1), res.rho.cpu().numpy(), res.batch_size)
    return f


def test_served_results_equal_alone(srv_mod):
    reqs = _requests(srv_mod, 14, seed=701, nmin=1_000, nmax=60_000)
    served, alone = {}, {}
    srv = srv_mod.Server(ngmax=NGMAX, slots=3, max_batch_particles=120_000)
    try:
        res = srv_mod.replay(srv, reqs, on_result=_grab(served))
    finally:
        srv.close()
    assert len(res) == len(reqs) and not srv.errors
    assert max(v[3] for v in served.values()) > 1, "no request was batched with another"
    srv_mod.replay_plain(reqs, ngmax=NGMAX, on_result=_grab(alone))
    for r in reqs:
        a, b = served[r.rid], alone[r.rid]
        assert np.array_equal(a[0], b[0]), f"request {r.rid}: counts"
        assert np.array_equal(a[1], b[1]), f"request {r.rid}: lists"
        assert np.array_equal(a[2].view(np.int32), b[2].view(np.int32)), f"request {r.rid}: densities"
    assert all(x.latency >= 0 for x in res)


def test_admission_waits_for_memory(srv_mod):
    # a budget of about two of these requests: at most two are ever in flight
    reqs = _requests(srv_mod, 8, seed=702, nmin=20_000, nmax=30_000)
    per = srv_mod.request_bytes(30_000, NGMAX)
    srv = srv_mod.Server(ngmax=NGMAX, slots=4, hbm_budget=2 * per + per // 2)
    inflight = []
    try:
        out = srv_mod.replay(srv, reqs, on_result=lambda r: inflight.append(
            srv.budget - srv._free_bytes))
    finally:
        srv.close()
    assert len(out) == len(reqs)
    assert max(inflight) <= srv.budget
    assert max(r.batch_size for r in out) <= 2


def test_oversized_request_is_refused(srv_mod):
    srv = srv_mod.Server(ngmax=NGMAX, slots=1, hbm_budget=1 << 24)
    try:
        r = _requests(srv_mod, 1, seed=703, nmin=100_000, nmax=100_001)[0]
        with pytest.raises(ValueError):
            srv.submit(r)
    finally:
        srv.close()


def test_a_bad_request_fails_alone(srv_mod):
    reqs = _requests(srv_mod, 6, seed=704, nmin=2_000, nmax=20_000)
    reqs[3].x[5] = float("nan")  # pinned host copy: poisoned input
    served, alone = {}, {}
    errors = {}

    def grab(res):
        if res.error is not None:
            errors[res.rid] = res.error
        else:
            _grab(served)(res)
    srv = srv_mod.Server(ngmax=NGMAX, slots=1, max_batch_particles=200_000)
    try:
        out = srv_mod.replay(srv, reqs, on_result=grab)
    finally:
        srv.close()
    assert len(out) == len(reqs) and not srv.errors
    assert set(errors) == {3} and "non-finite" in errors[3]
    good = [r for r in reqs if r.rid != 3]
    srv_mod.replay_plain(good, ngmax=NGMAX, on_result=_grab(alone))
    for r in good:
        a, b = served[r.rid], alone[r.rid]
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert np.array_equal(a[2].view(np.int32), b[2].view(np.int32))


def test_batches_on_different_slots_overlap_on_the_device(srv_mod):
    # continuous batching, not a queue: with requests arriving while others
    # run, batches of different slots are on the GPU at the same time (CUDA
    # event spans on the slots' streams)
    reqs = _requests(srv_mod, 24, seed=705, nmin=50_000, nmax=400_000, spread=0.02)
    srv = srv_mod.Server(ngmax=NGMAX, slots=3, max_batch_particles=500_000)
    try:
        out = srv_mod.replay(srv, reqs)
        tl = list(srv.timeline)
    finally:
        srv.close()
    assert len(out) == len(reqs) and not srv.errors
    assert len({slot for _, slot, _, _, _ in tl}) >= 2
    overlaps = [(a[0], b[0]) for i, a in enumerate(tl) for b in tl[i + 1:]
                if a[1] != b[1] and a[2] < b[3] and b[2] < a[3]]
    assert overlaps, f"no two batches of different slots overlapped on the device: {tl}"


def test_slot_trees_stay_charged_to_the_budget(srv_mod):
    # a slot keeps its tree after its batch: the budget accounts for it until
    # the tree is freed, and in-flight plus kept bytes never exceed the budget
    reqs = _requests(srv_mod, 10, seed=706, nmin=10_000, nmax=40_000)
    srv = srv_mod.Server(ngmax=NGMAX, slots=2)
    seen = []
    try:
        srv_mod.replay(srv, reqs, on_result=lambda r: seen.append(srv.budget - srv._free_bytes))
        kept = sum(srv._slot_tree)
        assert kept > 0 and srv.budget - srv._free_bytes == kept
    finally:
        srv.close()
    assert max(seen) <= srv.budget
