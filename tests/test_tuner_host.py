"""Host-side logic of the autotuner: the classes it tunes per are computed
from the data (set size and the spread of h), no GPU involved."""
import numpy as np

from paper_1910_02639_gb300 import workloads as wl


def test_tuner_classes_are_data_driven():
    from paper_1910_02639_gb300.autotune import set_class, size_class, spread_class
    assert size_class(1000) == 6 and size_class(3161) == 6 and size_class(3163) == 7
    assert spread_class(np.full(100, 0.3)) == 0
    assert spread_class(wl.evrard(20_000, seed=1).h) == 1
    assert spread_class(wl.plummer(20_000, seed=2).h) == 2
    assert set_class(wl.uniform_cube(5000, seed=3)) == (7, 0)


def test_list_checksum_semantics_on_cpu():
    """The checksum the batched and serving benchmarks compare: only the
    written part of each row counts, the order within a row counts, and the
    block size it works in does not change it."""
    import torch
    from paper_1910_02639_gb300.batch import list_checksum
    rng = np.random.default_rng(4)
    n, g = 1000, 8
    cnt = torch.from_numpy(rng.integers(0, 12, n).astype(np.int32))
    nb = torch.from_numpy(rng.integers(0, n, n * g).astype(np.int32))
    ref = list_checksum(nb, cnt, g)
    assert all(list_checksum(nb, cnt, g, chunk_rows=c) == ref for c in (1, 7, 64, 1 << 17))
    # entries past min(count, g) are ignored
    nb2 = nb.clone().view(n, g)
    for i in range(n):
        nb2[i, min(int(cnt[i]), g):] = -5
    assert list_checksum(nb2.view(-1), cnt, g) == ref
    # swapping two written entries of a row changes it
    i = int(np.nonzero(cnt.numpy() >= 2)[0][0])
    nb3 = nb.clone().view(n, g)
    if nb3[i, 0] != nb3[i, 1]:
        nb3[i, 0], nb3[i, 1] = nb3[i, 1].clone(), nb3[i, 0].clone()
        assert list_checksum(nb3.view(-1), cnt, g) != ref
