"""The library CPU sorts timed as the benchmark's CPU baseline (std::stable_sort, std::sort, and a
chunked parallel std::sort with pairwise merges) return the sorted keys. CPU only."""
import numpy as np
import pytest

from oracle import oracle as O
import workloads as W


@pytest.mark.parametrize("algo,threads", [("stable_sort", 1), ("sort", 1), ("parallel", 1),
                                          ("parallel", 3), ("parallel", 8)])
def test_cpu_sorts_return_the_sorted_keys(algo, threads):
    rs = np.random.RandomState(3)
    for keys in (W.lognormal_dup_f32(100_003, 2), rs.standard_normal(50_001),
                 W.gauss_mix_u64(70_001, 3)[0], np.zeros(0, np.float32), np.ones(5, np.float32)):
        out, dt = O.cpu_sort(keys, algo, threads)
        assert dt >= 0.0
        np.testing.assert_array_equal(out, np.sort(keys))
