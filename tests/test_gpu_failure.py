"""Failure detection without a GPU fault: the library's bounded device-side wait, run on a flag that
nothing sets, gives up after its limit and reports NNSORT_E_TIMEOUT to the host; the context stays
usable and the next sort is correct. Nothing faults, traps or hangs."""
import time

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)
import paper_1907_08817_gb300 as nns  # noqa: E402


def test_bounded_wait_expires_and_context_stays_usable():
    t0 = time.perf_counter()
    assert nns.selftest_wait(2000) == -6  # NNSORT_E_TIMEOUT
    assert time.perf_counter() - t0 < 5.0
    assert nns.selftest_wait(1) == -6
    keys = W.lognormal_dup_f32(200_000, 5, sigma=2.0)
    dk = torch.from_numpy(keys).cuda()
    f, _ = nns.train(dk, layers=1, h1=16, h2=0, sample_n=2000, steps=30, seed=0)
    nns.sort(dk, None, f)
    np.testing.assert_array_equal(dk.cpu().numpy().view(np.uint32),
                                  np.sort(keys, kind="stable").view(np.uint32))
    assert nns.stream_status() == 0
