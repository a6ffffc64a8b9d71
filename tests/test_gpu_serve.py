"""Serving with continuous batching (nnsort_server_*): each request's result is the same whether it is
served alone or in a mix with others, admission honours the HBM budget, FIFO mode agrees."""
import numpy as np
import pytest

from helpers import bits, stats_core
from oracle import oracle as orc
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)
import paper_1907_08817_gb300 as nns  # noqa: E402

TRAIN = dict(layers=2, h1=32, h2=32, sample_n=2000, steps=50, batch=0, lr=1e-2)


def _alone(keys: np.ndarray, seed: int):
    dk = torch.from_numpy(keys.copy()).cuda()
    model, _ = nns.train(dk, seed=seed, **{**TRAIN, "sample_n": min(TRAIN["sample_n"], keys.shape[0])})
    st = nns.sort(dk, None, model)
    return dk.cpu().numpy(), st


@pytest.mark.parametrize("mode", ["batched", "fifo"])
def test_server_results_equal_alone_and_in_the_mix(mode):
    reqs = W.serving_requests(count=20, seed=5, lo=10_000, hi=300_000, rate_per_s=1e6)
    arrays = [r["keys"].copy() for r in reqs]
    kw = dict(workers=2, max_batch=8) if mode == "batched" else dict(workers=1, max_batch=1)
    # a budget of a few requests: later arrivals wait for memory to free up
    with nns.Server(hbm_budget=120 << 20, train=TRAIN, **kw) as srv:
        tickets = [srv.submit(a, seed=i) for i, a in enumerate(arrays)]
        results = [srv.wait(t) for t in tickets]
    for i, r in enumerate(reqs):
        want, _ = orc.stable_sort(r["keys"])
        np.testing.assert_array_equal(bits(arrays[i]), bits(want))
        out, st = _alone(r["keys"], i)
        np.testing.assert_array_equal(bits(out), bits(arrays[i]))
        st_mix, lat = results[i]
        assert stats_core(st_mix) == stats_core(st)
        assert lat > 0


def test_server_budget_and_payload():
    keys = W.uniform_f32(200_000, 3).astype(np.float64)
    payload = np.arange(keys.shape[0], dtype=np.int32)
    with nns.Server(hbm_budget=1 << 20, train=TRAIN) as srv:  # smaller than one request
        with pytest.raises(nns.NNSortError) as ei:
            srv.submit(keys)
        assert ei.value.status == -4
    k2, p2 = keys.copy(), payload.copy()
    with nns.Server(train=TRAIN) as srv:
        t = srv.submit(k2, p2, seed=7)
        srv.wait(t)
    wk, wp = orc.stable_sort(keys, payload)
    np.testing.assert_array_equal(bits(k2), bits(wk))
    np.testing.assert_array_equal(p2, wp)
