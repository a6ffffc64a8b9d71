"""The paper's experiments on the device path, at sizes the oracle finishes: the changing
distribution of Exp-3 (a model trained on uniform keys sorting noisy inputs), the uniform uint64
stand-in for Exp-2's QuickDraw key-ids (also at its full 50,426,265 keys), and the paper's own
training recipe (Sec. Experimental Study: hidden layers of 2, 6 and 1 neurons, Huber loss of Eq.
(loss), batch 128, Adam lr 1e-3). Sorts are bit-exact to the oracle given the device's positions."""
import numpy as np
import pytest

from helpers import bits, from_dev, oracle_model, stats_core, to_dev
from oracle import oracle as orc
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)
import paper_1907_08817_gb300 as nns  # noqa: E402


def _parity(keys, model, precision="fp32", eps=3, tau=1024):
    dk, kt = to_dev(keys)
    slots, _ = nns.predict(dk, model, precision=precision, key_type=kt, want_y=False)
    L, _, _ = orc.nm_split(keys.shape[0])
    st = nns.sort(dk, None, model, precision=precision, eps=eps, tau=tau, key_type=kt)
    ok, _, ost, _ = orc.nnsort(keys, slots.cpu().numpy().astype(np.uint32), L, eps, tau)
    np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(ok))
    assert stats_core(st) == stats_core(ost)
    return st


def test_shift_model_trained_on_uniform_sorts_noisy_inputs():
    n = 300_000
    dtrain = torch.from_numpy(W.uniform_f32(1_000_000, 0)).cuda()
    f, _ = nns.train(dtrain, layers=1, h1=32, h2=0, sample_n=10_000, steps=100, lr=1e-2, seed=0)
    # the device model's positions are the oracle model's (same parameters, binary32 forward)
    om = oracle_model(f)
    sig = {}
    for noise in (0.0, 0.45):
        keys = W.shift_mix_f32(n, noise, seed=6)
        oslots, _ = orc.predict_slots(keys, om)
        dk, _ = to_dev(keys)
        slots, _ = nns.predict(dk, f, want_y=False)
        np.testing.assert_array_equal(slots.cpu().numpy().astype(np.uint32), oslots)
        st = _parity(keys, f)
        sig[noise] = st["sigma"][0]
    # noise crowds keys into positions the uniform model spreads thinly: more first-round conflicts
    assert sig[0.45] > sig[0.0] + 0.02, sig


@pytest.mark.parametrize("precision", ["fp32", "pwl"])
def test_uniform_u64_standin_small_parity(precision):
    keys = W.uniform_u64(250_000, seed=7)
    dk, kt = to_dev(keys)
    f, _ = nns.train(dk, key_type=kt, layers=1, h1=32, h2=0, sample_n=2500, steps=100, lr=1e-2,
                     seed=0)
    _parity(keys, f, precision)


def test_uniform_u64_standin_full_size():
    n = W.QUICKDRAW_RECORDS
    keys = W.uniform_u64(n, seed=7)
    dk, kt = to_dev(keys)
    flip = torch.tensor(-(1 << 63), dtype=torch.int64, device=dk.device)
    ref = torch.sort(dk ^ flip).values
    f, _ = nns.train(dk, key_type=kt, layers=1, h1=32, h2=0, sample_n=n // 100, steps=100,
                     lr=1e-2, seed=0)
    sig = {}
    for precision in ("fp32", "pwl"):
        work = dk.clone()
        st = nns.sort(work, None, f, precision=precision, key_type=kt)
        assert torch.equal(work ^ flip, ref), precision
        sig[precision] = st["sigma"][0]
    # n m = 6.3e7 positions exceed binary32's 2^24 steps per binade, so the binary32 form maps runs of
    # neighbouring keys to one position; the compiled form resolves them
    assert sig["pwl"] < sig["fp32"] - 0.1, sig


def test_paper_training_recipe_tracks_binary64():
    keys = W.lognormal_dup_f32(1_000_000, 2, sigma=2.0)
    dk, _ = to_dev(keys)
    cfg = dict(layers=2, h1=2, h2=6, sample_n=20_000, steps=300, batch=128, lr=1e-3, seed=0)
    model, hist = nns.train(dk, loss="huber", huber_delta=0.01, **cfg)
    _, p64, ohist = orc.train(keys, translate=orc.ORDBITS, loss=orc.HUBER, huber_delta=0.01, **cfg)
    _, p = model.describe()
    assert abs(hist[0] - ohist[0]) <= 1e-5 * abs(ohist[0]) + 1e-8
    np.testing.assert_allclose(hist, ohist, rtol=2e-3, atol=1e-7)
    assert np.max(np.abs(p - p64)) <= 2e-3 * np.abs(p64).max()
    assert np.mean(hist[-50:]) < np.mean(hist[:50])
    # the trained 1-2-6-1 sorts bit-exactly given its positions
    _parity(keys[:200_000], model)
