"""The autotuner on the device: every candidate setting gives the same sorted output (checked inside
tune_gpu), the chosen setting lies in the space, and sorts that take the tuned setting from the
table still match the oracle bit for bit, per-iteration counts included."""
import numpy as np
import pytest

from helpers import bits, from_dev, lib_model, stats_core, to_dev
from oracle import oracle as orc
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)
import paper_1907_08817_gb300 as nns  # noqa: E402
from paper_1907_08817_gb300 import autotune as AT  # noqa: E402

SPACE = {"bucket_log2": (9, 12, 14), "polish_blocks": (1, 3), "eps": (1, 3)}


def test_tune_then_sort_with_tuned_setting(tmp_path, monkeypatch):
    path = str(tmp_path / "tuned.json")
    keys = W.lognormal_dup_f32(300_001, 11, sigma=2.0)
    om, _, _ = orc.train(keys, 1, 32, 0, orc.ORDBITS, sample_n=3000, steps=60, lr=1e-2, seed=1)
    f = lib_model(om)
    dk, kt = to_dev(keys)
    best, log = AT.tune_gpu([dk], [f], "fp32", space=SPACE, repeats=1, write=True, path=path)
    assert all(best[k] in v for k, v in SPACE.items())
    assert len(log) >= 4 and all(t > 0 for _, t in log)
    monkeypatch.setattr(AT, "TABLE", path)
    monkeypatch.setattr(AT.tuned_options, "__defaults__", (path,))
    assert AT.tuned_options(0, keys.shape[0], 1, 32, 0, "fp32") == best
    st = nns.sort(dk, None, f, eps="auto")
    assert st["bucket_log2"] == best["bucket_log2"] and st["eps"] == best["eps"]
    ok, _, ost, _ = orc.nnsort_model(keys, om, eps=best["eps"])
    np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(ok))
    assert stats_core(st) == stats_core(ost)


def test_tune_batch_with_payload():
    arrs, models = [], []
    for j, (_, a) in enumerate(W.batch_arrays(12, seed=9, lo=1000, hi=100_000)):
        om, _, _ = orc.train(a, 1, 16, 0, orc.ORDBITS, sample_n=max(100, a.shape[0] // 100),
                             steps=30, lr=1e-2, seed=j)
        arrs.append(a)
        models.append(lib_model(om))
    dks = [to_dev(a)[0] for a in arrs]
    pays = [torch.arange(a.shape[0], dtype=torch.int32, device="cuda") for a in arrs]
    best, _ = AT.tune_gpu(dks, models, "fp32", payloads=pays, space=SPACE, repeats=1)
    nns.sort_batch(dks, models, pays, **best)
    for a, dk, p in zip(arrs, dks, pays):
        wk, wp = orc.stable_sort(a, np.arange(a.shape[0], dtype=np.int32))
        np.testing.assert_array_equal(bits(from_dev(dk, a)), bits(wk))
        np.testing.assert_array_equal(p.cpu().numpy(), wp)
