"""BF16 tensor-core (tcgen05) forward pass inside the sort.

The model output is compared with a binary64 emulation of the same arithmetic (binary32 first
layer, BF16-rounded hidden activations and weights, exact products and second-layer bias, wide
accumulation); only the tensor core's FP32 accumulation order differs, so the tolerance is a few
binary32 ulps of the accumulated magnitude. Given the positions the BF16 path produced, the rest of the sort must match
the oracle bit for bit; displacement against the binary64 model is reported, not asserted."""
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


def _bf16(a: np.ndarray) -> np.ndarray:
    """Round binary32 values to BF16 (nearest, ties to even), returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _emulate(params: np.ndarray, h: int, x: np.ndarray, split: bool = False):
    p = params.astype(np.float64)
    W2 = p[2 * h:2 * h + h * h].reshape(h, h)
    b2 = p[2 * h + h * h:3 * h + h * h]
    W3 = p[3 * h + h * h:4 * h + h * h]
    b3 = p[4 * h + h * h]
    a = orc.mlp_layer1_f32(2, h, h, params, x)  # binary32 first layer (after the ReLU)
    W2b = _bf16(W2.astype(np.float32))
    if split:
        # a = hi + lo: hi = a truncated to BF16 (8 significant bits) times W2 in BF16, plus
        # lo = the exact binary32 rest rounded to FP16 times W2 in FP16
        hi = (a.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
        lo = (a.astype(np.float64) - hi).astype(np.float32).astype(np.float16).astype(np.float64)
        W2h = W2.astype(np.float32).astype(np.float16).astype(np.float64)
        z = hi @ W2b.T + lo @ W2h.T
        h1 = hi + lo
    else:
        h1 = _bf16(a)
        z = h1 @ W2b.T
    h2 = np.maximum(z + b2, 0)
    terms = np.abs(h2 * W3).sum(axis=1) + abs(b3)
    # b2 is accumulated by the tensor core with the products (as one more K-step of exact BF16
    # parts), so it belongs to the accumulated magnitude
    return h2 @ W3 + b3, terms, np.abs(h1) @ np.abs(W2b).T + np.abs(b2)


@pytest.mark.parametrize("h", [16, 32, 64])
@pytest.mark.parametrize("prec", ["bf16", "bf16x2"])
def test_bf16_forward_matches_emulation(h, prec):
    keys = W.lognormal_dup_f32(300_000, 31, sigma=2.0)
    om, _, _ = orc.train(keys, 2, h, h, orc.ORDBITS, sample_n=3000, steps=60, seed=h)
    f = lib_model(om)
    dk, _ = to_dev(keys)
    slots, y = nns.predict(dk, f, precision=prec)
    x = orc.translate_f32(keys, om.norm)
    ye, terms, zmag = _emulate(om.params, h, x, split=prec == "bf16x2")
    yg = y.cpu().numpy().astype(np.float64)
    W3 = np.abs(om.params[3 * h + h * h:4 * h + h * h].astype(np.float64))
    # tensor-core accumulation of z (<= 2 ulp of |z| terms) propagated through |W3|, plus the
    # binary32 output layer
    tol = 4 * 2.0 ** -23 * (zmag @ W3 + terms) + 1e-7
    assert np.all(np.abs(yg - ye) <= tol), float(np.max(np.abs(yg - ye) - tol))
    # displacement against the binary32 and binary64 models (reported)
    s32, _ = orc.predict_slots(keys, om)
    sg = slots.cpu().numpy().astype(np.int64)
    d = np.abs(sg - s32.astype(np.int64))
    print(f"H={h} {prec}: |slot - slot_fp32| mean {d.mean():.2f} max {d.max()}")


@pytest.mark.parametrize("h", [32, 64])
@pytest.mark.parametrize("prec", ["bf16", "bf16x2"])
def test_bf16_sort_matches_oracle_given_its_positions(h, prec):
    keys = W.lognormal_dup_f32(400_000, 41, sigma=2.0)
    payload = np.arange(keys.shape[0], dtype=np.int32)
    om, _, _ = orc.train(keys, 2, h, h, orc.ORDBITS, sample_n=4000, steps=80, seed=h)
    f = lib_model(om)
    dk, _ = to_dev(keys)
    slots, _ = nns.predict(dk, f, precision=prec, want_y=False)
    dp = torch.from_numpy(payload).cuda()
    st = nns.sort(dk, dp, f, precision=prec)
    L, _, _ = orc.nm_split(keys.shape[0])
    ok, op, ost, _ = orc.nnsort(keys, slots.cpu().numpy().astype(np.uint32), L, 3, 1024, payload)
    np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(ok))
    np.testing.assert_array_equal(dp.cpu().numpy(), op)
    assert stats_core(st) == stats_core(ost)


def test_bf16_without_hidden_to_hidden_layer():
    keys = torch.rand(5000, device="cuda")
    nm = orc.make_norm(keys.cpu().numpy(), np.arange(5000, dtype=np.uint64), orc.VALUE)
    # one hidden layer: nothing runs on the tensor cores, BF16 is the binary32 path
    one = lib_model(orc.Model(1, 32, 0, nm, orc.init_params(1, 32, 0, 0)))
    s32, y32 = nns.predict(keys, one, precision="fp32")
    s16, y16 = nns.predict(keys, one, precision="bf16")
    assert torch.equal(s32, s16) and torch.equal(y32, y16)
    # hidden widths below one MMA tile (16) are not built for the tensor path
    tiny = lib_model(orc.Model(2, 4, 4, nm, orc.init_params(2, 4, 4, 0)))
    with pytest.raises(nns.NNSortError) as ei:
        nns.sort(keys, None, tiny, precision="bf16")
    assert ei.value.status == -7


def test_split_bf16_resolves_f_like_binary32():
    """The split form carries ~16 significant bits of each activation: F(x) takes about as many
    distinct values over the keys as the binary32 model, where plain BF16 collapses runs of
    neighbouring keys onto one value."""
    keys = np.sort(W.lognormal_f32(400_000, 51, sigma=2.0))
    om, _, _ = orc.train(keys, 2, 64, 64, orc.ORDBITS, sample_n=4000, steps=80, seed=3)
    f = lib_model(om)
    dk, _ = to_dev(keys)
    distinct = {}
    for prec in ("fp32", "bf16", "bf16x2"):
        _, y = nns.predict(dk, f, precision=prec)
        distinct[prec] = int(torch.unique(y).numel())
    assert distinct["bf16x2"] >= 0.9 * distinct["fp32"]
    assert distinct["bf16x2"] > 2 * distinct["bf16"]


@pytest.mark.parametrize("prec", ["bf16", "bf16x2"])
def test_batched_tensor_core_forms_match_the_oracle_given_single_array_positions(prec):
    """Arrays of a batch, each with its own 1-64-64-1 model, run through the batched tensor-core
    kernel (one W2 per array, reloaded when a block's sub-tile changes array). Its positions equal
    the single-array kernel's for the same model (same per-row arithmetic), so every array's output,
    payload and per-round counts must equal the oracle's procedure given those positions."""
    arrs = [a for _, a in W.batch_arrays(7, seed=44, lo=20_000, hi=150_000)]
    models, slots = [], []
    for j, a in enumerate(arrs):
        om, _, _ = orc.train(a, 2, 64, 64, orc.ORDBITS, sample_n=1000, steps=20, seed=j)
        f = lib_model(om)
        models.append(f)
        s, _ = nns.predict(to_dev(a)[0], f, precision=prec, want_y=False)
        slots.append(s.cpu().numpy().astype(np.uint32))
    dks = [to_dev(a)[0] for a in arrs]
    dps = [torch.arange(a.shape[0], dtype=torch.int32, device="cuda") for a in arrs]
    sts = nns.sort_batch(dks, models, dps, precision=prec, eps=3, bucket_log2=12, polish_blocks=2)
    for a, s, dk, dp, st in zip(arrs, slots, dks, dps, sts):
        L, _, _ = orc.nm_split(a.shape[0])
        ok, op, ost, _ = orc.nnsort(a, s, L, 3, 1024, np.arange(a.shape[0], dtype=np.int32))
        np.testing.assert_array_equal(bits(from_dev(dk, a)), bits(ok))
        np.testing.assert_array_equal(dp.cpu().numpy(), op)
        assert stats_core(st) == stats_core(ost)
