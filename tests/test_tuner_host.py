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
