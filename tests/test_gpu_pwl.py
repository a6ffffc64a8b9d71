"""NNSORT_PREC_PWL on the device: positions equal those of the binary64 model (oracle translate and
forward pass in binary64, position rounded from binary64) except where rounding lands within a few
ulps of a half-position (at most one position apart, rare); sorts given those positions match the
oracle bit for bit (keys, payload, per-iteration counts, fates); finer positions than binary32."""
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


def _slots64(keys, om, m=1.25):
    """Positions of the binary64 model: round-half-up of F * n * m, F <= 0 -> 0, clamped to L - 1."""
    n = keys.shape[0]
    L, nm_hi, nm_lo = orc.nm_split(n, m)
    y = orc.mlp_forward_f64(om.layers, om.h1, om.h2, om.params, orc.translate_f64(keys, om.norm))
    nm = float(np.float32(nm_hi)) + float(np.float32(nm_lo))
    s = np.floor(np.minimum(y, 1.0) * nm + 0.5)
    s = np.where(y > 0, s, 0)
    return np.clip(s, 0, L - 1).astype(np.int64), L


def _case(case):
    payload = None
    if case == "ln_f32_2l":
        keys = W.lognormal_dup_f32(400_003, 2, sigma=2.0)
        om, _, _ = orc.train(keys, 2, 32, 32, orc.ORDBITS, sample_n=4000, steps=80, seed=1)
    elif case == "u_f32_value_1l":
        keys = W.uniform_f32(300_000, 0)
        om, _, _ = orc.train(keys, 1, 32, 0, orc.VALUE, sample_n=3000, steps=100, seed=0)
    elif case == "gm_u64_kv":
        keys, payload = W.gauss_mix_u64(250_000, 3)
        om, _, _ = orc.train(keys, 2, 16, 16, orc.ORDBITS, sample_n=3000, steps=60, seed=2)
    else:  # f64 keys, VALUE translate
        keys = W.normal_f32(200_000, 6).astype(np.float64) * 1e3
        om, _, _ = orc.train(keys, 1, 16, 0, orc.VALUE, sample_n=3000, steps=80, seed=4)
    return keys, payload, om


@pytest.mark.parametrize("case", ["ln_f32_2l", "u_f32_value_1l", "gm_u64_kv", "f64_value_1l"])
def test_pwl_positions_are_the_binary64_models(case):
    keys, payload, om = _case(case)
    f = lib_model(om)
    dk, kt = to_dev(keys)
    slots, _ = nns.predict(dk, f, precision="pwl", key_type=kt, want_y=False)
    sp = slots.cpu().numpy()
    s64, L = _slots64(keys, om)
    d = np.abs(sp - s64)
    assert d.max() <= 1, int(d.max())
    assert (d != 0).mean() <= 1e-4, float((d != 0).mean())


@pytest.mark.parametrize("case", ["ln_f32_2l", "gm_u64_kv"])
def test_pwl_sort_matches_oracle_given_its_positions(case):
    keys, payload, om = _case(case)
    f = lib_model(om)
    dk, kt = to_dev(keys)
    slots, _ = nns.predict(dk, f, precision="pwl", key_type=kt, want_y=False)
    L, _, _ = orc.nm_split(keys.shape[0])
    dp = None if payload is None else torch.from_numpy(payload).cuda()
    st, fate = nns.sort(dk, dp, f, precision="pwl", fate=True, key_type=kt)
    ok, op, ost, ofate = orc.nnsort(keys, slots.cpu().numpy().astype(np.uint32), L, 3, 1024, payload,
                                    want_fate=True)
    np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(ok))
    if payload is not None:
        np.testing.assert_array_equal(dp.cpu().numpy(), op)
    assert stats_core(st) == stats_core(ost)
    np.testing.assert_array_equal(fate.cpu().numpy(), ofate)


def test_pwl_resolves_more_positions_than_binary32():
    """At 2^24 keys binary32 translate and forward pass cannot separate neighbouring keys; the compiled
    form (about 48 significant bits per key) can, so fewer keys conflict in the first iteration."""
    n = 1 << 24
    keys = W.lognormal_dup_f32(n, 2, sigma=2.0)
    dk = torch.from_numpy(keys).cuda()
    f, _ = nns.train(dk, layers=2, h1=32, h2=32, sample_n=n // 100, steps=100, batch=65536, seed=0)
    sig = {}
    for prec in ("fp32", "pwl"):
        work = dk.clone()
        st = nns.sort(work, None, f, precision=prec)
        sig[prec] = st["sigma"][0]
        assert torch.equal(work, torch.sort(dk).values)
    assert sig["pwl"] < sig["fp32"] - 0.02, sig


def test_pwl_batch_is_unsupported():
    arrs = [W.uniform_f32(5000, j) for j in range(2)]
    oms = [orc.train(a, 1, 8, 0, orc.VALUE, sample_n=500, steps=20, seed=j)[0] for j, a in enumerate(arrs)]
    with pytest.raises(nns.NNSortError) as ei:
        nns.sort_batch([to_dev(a)[0] for a in arrs], [lib_model(om) for om in oms], precision="pwl")
    assert ei.value.status == -7
