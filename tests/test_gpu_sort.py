"""GPU parity of the NN-sort pipeline against the CPU oracle, through the C ABI.

Positions, outputs, per-iteration counts and per-row fates are integer results and must match the
oracle bit for bit; the sort output is the stable order of the keys, bit for bit."""
import numpy as np
import pytest

from helpers import bits, from_dev, lib_model, oracle_model, stats_core, to_dev
from oracle import oracle as orc
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)
import paper_1907_08817_gb300 as nns  # noqa: E402


def _rand_model(dtype_code, keys, layers, h1, h2, translate, seed=0, S=2000):
    rows, nm, _, _ = orc.sample_labels(keys, S, seed, translate)
    return orc.Model(layers, h1, h2, nm, orc.init_params(layers, h1, h2, seed))


def _trained(keys, layers, h1, h2, translate, S=2000, steps=100, seed=0):
    m, _, _ = orc.train(keys, layers, h1, h2, translate, sample_n=S, steps=steps, lr=1e-2, seed=seed)
    return m


# ---------------------------------------------------------------------------- prediction (a3, a4)
@pytest.mark.parametrize("case", ["u_f32_value", "ln_f32_ordbits_2l", "gm_u64", "n_f64_value",
                                  "ln_f32_64x64"])
def test_predict_positions_bit_exact(case):
    if case == "u_f32_value":
        keys, om = W.uniform_f32(100_003, 1), None
        om = _trained(keys, 1, 32, 0, orc.VALUE)
    elif case == "ln_f32_ordbits_2l":
        keys = W.lognormal_dup_f32(77_777, 2, sigma=2.0)
        om = _trained(keys, 2, 16, 16, orc.ORDBITS, steps=50)
    elif case == "gm_u64":
        keys, _ = W.gauss_mix_u64(50_001, 3)
        om = _trained(keys, 2, 32, 32, orc.ORDBITS, steps=30)
    elif case == "n_f64_value":
        keys = W.normal_f32(40_000, 4).astype(np.float64) * 1e3
        om = _trained(keys, 1, 8, 0, orc.VALUE)
    else:
        keys = W.lognormal_dup_f32(20_000, 5, sigma=2.0)
        om = _rand_model(orc.F32, keys, 2, 64, 64, orc.ORDBITS)
    f = lib_model(om)
    dk, kt = to_dev(keys)
    for m in (1.25, 2.0):
        slots, y = nns.predict(dk, f, m=m, key_type=kt)
        om_slots, om_y = orc.predict_slots(keys, om, m)
        np.testing.assert_array_equal(slots.cpu().numpy().astype(np.uint32), om_slots)
        np.testing.assert_array_equal(y.cpu().numpy().view(np.uint32), om_y.view(np.uint32))


# ---------------------------------------------------------------------------- injected positions
def _check_injected(keys, slots, L, eps, tau, payload=None, bucket_log2=0):
    dk, kt = to_dev(keys)
    dp = None if payload is None else torch.from_numpy(payload).cuda()
    ds = torch.from_numpy(slots.astype(np.uint32).view(np.int32)).cuda()
    st, fate = nns.sort(dk, dp, None, eps=eps, tau=tau, slots=ds, fate=True, key_type=kt,
                        bucket_log2=bucket_log2)
    ok, op, ost, ofate = orc.nnsort(keys, slots, L, eps, tau, payload, want_fate=True)
    np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(ok))
    if payload is not None:
        np.testing.assert_array_equal(dp.cpu().numpy(), op)
    assert stats_core(st) == stats_core(ost)
    np.testing.assert_array_equal(fate.cpu().numpy(), ofate)
    return st


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 1023, 4097, 65_537, 300_001])
def test_injected_positions_match_oracle(n):
    rs = np.random.RandomState(n)
    keys = W.normal_f32(n, n)
    L, _, _ = orc.nm_split(n)
    # positions roughly following the key order, with noise, collisions and out-of-order picks
    rank = np.argsort(np.argsort(keys, kind="stable"), kind="stable")
    slots = np.clip((rank * 1.25 + rs.randint(-3, 4, n)).astype(np.int64), 0, L - 1)
    slots[rs.rand(n) < 0.05] = rs.randint(0, L, max(1, int((rs.rand(n) < 0.05).sum())))[:1]
    for eps, tau in ((3, 0), (1, 0), (4, 7), (3, n + 1)):
        _check_injected(keys, slots.astype(np.uint32), L, eps, tau,
                        payload=np.arange(n, dtype=np.int32))


@pytest.mark.parametrize("kind", ["few_distinct", "far_outliers", "spread", "u64_spread"])
def test_bucket_sort_paths(kind):
    """Each bucket is sorted whole: by one counting pass over bins of its key range, or by radix
    sort when a bin crowds (few distinct keys, or a few far outliers that stretch the range).
    Positions follow the key order (buckets of ~3,300 keys at 4,096 positions), with noise."""
    n = 300_000
    rs = np.random.RandomState(11)
    if kind == "few_distinct":
        keys = rs.randint(0, 40, n).astype(np.float32)
    elif kind == "far_outliers":
        keys = W.uniform_f32(n, 12)
        far = rs.rand(n) < 0.002
        keys[far] = np.float32(3.0e38)
    elif kind == "spread":
        keys = W.lognormal_dup_f32(n, 13, sigma=2.0)
    else:
        keys = W.uniform_u64(n, 14)
    L, _, _ = orc.nm_split(n)
    rank = np.argsort(np.argsort(keys, kind="stable"), kind="stable")
    slots = np.clip((rank * 1.25 + rs.randint(-40, 41, n)).astype(np.int64), 0, L - 1)
    if kind == "far_outliers":  # the outliers land in random buckets and stretch their key range
        slots[far] = rs.randint(0, L, int(far.sum()))
    payload = np.arange(n, dtype=np.int32)
    for eps in (1, 3):
        _check_injected(keys, slots.astype(np.uint32), L, eps, 0, payload=payload, bucket_log2=12)
        _check_injected(keys, slots.astype(np.uint32), L, eps, 0, bucket_log2=12)


def test_injected_degenerate_maps():
    n = 20_000
    keys = W.uniform_f32(n, 9)
    L, _, _ = orc.nm_split(n)
    # every key on one position: each round stores one element, the rest is the leftover
    st = _check_injected(keys, np.full(n, 5, np.uint32), L, 3, 0, np.arange(n, dtype=np.int32))
    assert st["w_size"] == [n, n - 1, n - 2, n - 3]
    # reverse order: every stored element but the first of each o_i is out of order
    rank = np.argsort(np.argsort(keys, kind="stable"), kind="stable")
    _check_injected(keys, ((n - 1 - rank) * 5 // 4).astype(np.uint32), L, 3, 0)
    # random positions over the whole range (non-monotone everywhere: seam repair)
    rs = np.random.RandomState(3)
    _check_injected(keys, rs.randint(0, L, n).astype(np.uint32), L, 3, 10,
                    np.arange(n, dtype=np.int32))


def test_large_seam_repair_runs_as_multi_block_sort():
    """Positions unrelated to key order put violators across the whole output; the repair is
    then larger than one block handles and runs as a multi-block radix sort."""
    rs = np.random.RandomState(13)
    for n, dt in ((300_000, np.float32), (200_000, np.uint64)):
        keys = (W.normal_f32(n, 14) if dt == np.float32
                else rs.randint(0, 2 ** 62, n, dtype=np.int64).astype(np.uint64))
        L, _, _ = orc.nm_split(n)
        slots = rs.randint(0, L, n).astype(np.uint32)
        dk, kt = to_dev(keys)
        ds = torch.from_numpy(slots.view(np.int32)).cuda()
        st = nns.sort(dk, None, None, slots=ds, key_type=kt)
        ok, _, ost, _ = orc.nnsort(keys, slots, L, 3, 1024)
        np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(ok))
        assert stats_core(st) == stats_core(ost)
        assert st["repaired"] > 65_536
    # a random (untrained) two-layer model is non-monotone: same outcome through the model path
    keys = W.lognormal_dup_f32(500_000, 15, sigma=2.0)
    om = _rand_model(orc.F32, keys, 2, 16, 16, orc.ORDBITS, seed=5)
    dk, _ = to_dev(keys)
    st = nns.sort(dk, None, lib_model(om))
    ok, _, ost, _ = orc.nnsort_model(keys, om)
    np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(ok))
    assert stats_core(st) == stats_core(ost)


def test_injected_small_buckets_and_oversized():
    rs = np.random.RandomState(11)
    n = 120_000
    keys = W.lognormal_f32(n, 12, sigma=1.0)
    L, _, _ = orc.nm_split(n)
    rank = np.argsort(np.argsort(keys, kind="stable"), kind="stable")
    slots = (rank * 5 // 4).astype(np.int64)
    # a crowded stretch: 40% of the keys squeezed into 64 positions -> oversized buckets
    crowd = rs.rand(n) < 0.4
    slots[crowd] = 1000 + (slots[crowd] % 64)
    st = _check_injected(keys, slots.astype(np.uint32), L, 3, 0, np.arange(n, dtype=np.int32),
                         bucket_log2=9)
    assert st["oversized_buckets"] >= 1


# ---------------------------------------------------------------------------- model-driven sorts
@pytest.mark.parametrize("case", ["c1_uniform", "lognormal_dup", "u64_kv", "f64", "two_layer"])
def test_model_sort_matches_oracle(case):
    payload = None
    if case == "c1_uniform":
        keys = W.uniform_f32(1_000_000, 0)
        om = _trained(keys, 1, 32, 0, orc.VALUE, S=10_000)
    elif case == "lognormal_dup":
        keys = W.lognormal_dup_f32(500_000, 2, sigma=2.0)
        om = _trained(keys, 1, 32, 0, orc.ORDBITS, S=5000)
    elif case == "u64_kv":
        keys, payload = W.gauss_mix_u64(300_000, 3)
        om = _trained(keys, 2, 16, 16, orc.ORDBITS, S=5000, steps=60)
    elif case == "f64":
        keys = W.normal_f32(200_000, 6).astype(np.float64)
        om = _trained(keys, 1, 16, 0, orc.VALUE, S=3000)
    else:
        keys = W.exponential_f32(250_000, 7)
        om = _trained(keys, 2, 8, 8, orc.ORDBITS, S=3000, steps=80)
    f = lib_model(om)
    dk, kt = to_dev(keys)
    dp = None if payload is None else torch.from_numpy(payload).cuda()
    st, fate = nns.sort(dk, dp, f, fate=True, key_type=kt)
    ok, op, ost, ofate = orc.nnsort_model(keys, om, payload=payload, want_fate=True)
    np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(ok))
    if payload is not None:
        np.testing.assert_array_equal(dp.cpu().numpy(), op)
    assert stats_core(st) == stats_core(ost)
    np.testing.assert_array_equal(fate.cpu().numpy(), ofate)
    # and without the trace (rows not carried): same output and counts
    dk2, _ = to_dev(keys)
    st2 = nns.sort(dk2, None, f, key_type=kt)
    np.testing.assert_array_equal(bits(from_dev(dk2, keys)), bits(ok))
    assert stats_core(st2) == stats_core(ost)


def test_edge_keys_and_empty():
    v = np.array([np.inf, -0.0, 0.0, -np.inf, 1.0, -1.0, 0.0, -0.0, 3e38, -3e38, 1e-45, -1e-45] * 50,
                 dtype=np.float32)
    rs = np.random.RandomState(0)
    v = v[rs.permutation(v.shape[0])]
    om = _rand_model(orc.F32, v, 1, 8, 0, orc.ORDBITS, S=100)
    f = lib_model(om)
    dk, _ = to_dev(v)
    dp = torch.arange(v.shape[0], dtype=torch.int32, device="cuda")
    st = nns.sort(dk, dp, f)
    ok, op, ost, _ = orc.nnsort_model(v, om, payload=np.arange(v.shape[0], dtype=np.int32))
    np.testing.assert_array_equal(bits(from_dev(dk, v)), bits(ok))
    np.testing.assert_array_equal(dp.cpu().numpy(), op)
    assert stats_core(st) == stats_core(ost)
    # all-equal keys
    eq = np.full(70_000, 2.5, dtype=np.float32)
    om2 = _rand_model(orc.F32, eq, 1, 8, 0, orc.VALUE, S=100)
    dk, _ = to_dev(eq)
    dp = torch.arange(eq.shape[0], dtype=torch.int32, device="cuda")
    st = nns.sort(dk, dp, lib_model(om2))
    assert np.array_equal(dp.cpu().numpy(), np.arange(eq.shape[0]))
    # empty and single
    e = torch.empty(0, dtype=torch.float32, device="cuda")
    assert nns.sort(e, None, f)["n"] == 0
    one = torch.tensor([4.0], device="cuda")
    nns.sort(one, None, f)
    assert one.item() == 4.0


def test_nan_keys_rejected_input_untouched():
    keys = W.uniform_f32(10_000, 3)
    om = _rand_model(orc.F32, keys, 1, 8, 0, orc.VALUE, S=100)
    keys[777] = np.nan
    dk, _ = to_dev(keys)
    before = dk.clone()
    with pytest.raises(nns.NNSortError) as ei:
        nns.sort(dk, None, lib_model(om))
    assert ei.value.status == -2
    assert torch.equal(dk.view(torch.int32), before.view(torch.int32))


def test_invalid_arguments():
    keys = torch.rand(100, device="cuda")
    with pytest.raises(nns.NNSortError):
        nns.sort(keys, None, None)  # no model and no injected positions
    om = _rand_model(orc.F32, keys.cpu().numpy(), 1, 8, 0, orc.VALUE, S=50)
    with pytest.raises(nns.NNSortError):
        nns.sort(keys, None, lib_model(om), eps=99)
    with pytest.raises(nns.NNSortError):
        nns.sort(keys.double(), None, lib_model(om))  # dtype differs from the model's


# ---------------------------------------------------------------------------- batch
def test_batch_equals_individual_sorts():
    arrs, models, oms = [], [], []
    for j, (kind, a) in enumerate(W.batch_arrays(24, seed=4, lo=1000, hi=200_000)):
        om = _trained(a, 1, 16, 0, orc.ORDBITS, S=max(100, a.shape[0] // 100), steps=50, seed=j)
        arrs.append(a)
        oms.append(om)
        models.append(lib_model(om))
    dks = [to_dev(a)[0] for a in arrs]
    sts = nns.sort_batch(dks, models)
    for a, om, dk, st in zip(arrs, oms, dks, sts):
        ok, _, ost, _ = orc.nnsort_model(a, om)
        np.testing.assert_array_equal(bits(from_dev(dk, a)), bits(ok))
        assert stats_core(st) == stats_core(ost)


def test_host_entry_point():
    keys = W.lognormal_dup_f32(100_000, 8, sigma=2.0)
    payload = np.arange(keys.shape[0], dtype=np.int32)
    om = _trained(keys, 1, 32, 0, orc.ORDBITS, S=1000)
    k2, p2 = keys.copy(), payload.copy()
    st = nns.sort_host(k2, p2, lib_model(om))
    ok, op, ost, _ = orc.nnsort_model(keys, om, payload=payload)
    np.testing.assert_array_equal(bits(k2), bits(ok))
    np.testing.assert_array_equal(p2, op)
    assert stats_core(st) == stats_core(ost)


# ---------------------------------------------------------------------------- tunables
def test_every_bucket_width_and_polish_occupancy():
    """Every (bucket_log2, polish_blocks) the autotuner may pick gives the oracle's output and
    counts; at 2^14 positions per bucket the position table alone exceeds a third of an SM's shared
    memory, so fewer polish blocks share the SM."""
    keys = W.lognormal_dup_f32(200_003, 12, sigma=2.0)
    om = _trained(keys, 1, 32, 0, orc.ORDBITS, S=2000, steps=60)
    f = lib_model(om)
    ok, _, ost, _ = orc.nnsort_model(keys, om)
    for wlog in range(9, 15):
        for pb in (1, 2, 3):
            dk, kt = to_dev(keys)
            st = nns.sort(dk, None, f, bucket_log2=wlog, polish_blocks=pb, key_type=kt)
            np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(ok))
            assert stats_core(st) == stats_core(ost)
            assert st["bucket_log2"] == wlog


# ---------------------------------------------------------------------------- seam ranges
def _expected_seam(keys: np.ndarray, slots: np.ndarray, wlog: int):
    """From the definition: concatenate the buckets, each sorted by key; a cut between positions
    p-1 and p is sound when max(out[:p]) <= min(out[p:]); the ranges to re-sort are the gaps of two
    or more elements between consecutive sound cuts. Returns (count, elements)."""
    n = keys.shape[0]
    out = keys[np.lexsort((keys, slots.astype(np.int64) >> wlog))].astype(np.float64)
    pm = np.maximum.accumulate(out)[:-1]           # max(out[:p]) for p = 1 .. n-1
    sm = np.minimum.accumulate(out[::-1])[::-1][1:]  # min(out[p:]) for p = 1 .. n-1
    cuts = np.concatenate(([0], 1 + np.nonzero(pm <= sm)[0], [n]))
    gaps = np.diff(cuts)
    big = gaps[gaps >= 2]
    return int(big.shape[0]), int(big.sum())


@pytest.mark.parametrize("n,moves,far", [(100_000, 0, False), (100_000, 40, False),
                                         (1_000_000, 300, False), (1_000_000, 300, True)])
def test_seam_repairs_exactly_the_unsound_ranges(n, moves, far):
    """Positions that follow the key order except for a few keys sent a little (or, with far=True,
    one key sent very far) across bucket boundaries: the repair touches exactly the ranges between
    consecutive sound cuts; a range longer than one block handles runs as the multi-block sort."""
    rs = np.random.RandomState(n + moves + far)
    keys = W.uniform_f32(n, 21)
    L, _, _ = orc.nm_split(n)
    rank = np.argsort(np.argsort(keys, kind="stable"), kind="stable")
    slots = (rank * 5 // 4).astype(np.int64)
    idx = rs.choice(n, moves, replace=False)
    slots[idx] += rs.randint(-6000, 6000, moves)
    if far:
        slots[np.argmin(keys)] = L - 1
    slots = np.clip(slots, 0, L - 1).astype(np.uint32)
    dk, kt = to_dev(keys)
    ds = torch.from_numpy(slots.view(np.int32)).cuda()
    st = nns.sort(dk, None, None, slots=ds, key_type=kt, bucket_log2=12)
    np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(np.sort(keys, kind="stable")))
    cnt, elems = _expected_seam(keys, slots, 12)
    assert (st["repair_ranges"], st["repaired"]) == (cnt, elems)
    if moves and not far:
        assert cnt >= 2
    if far:  # the smallest key in the last bucket: one range over nearly the whole array
        assert cnt == 1 and elems > n - 4096


def test_bucket_scans_on_many_blocks():
    """Arrays of more than one tile of buckets run the scans over buckets (the polish's carries per
    round, the seam's prefix maxima and suffix minima) on many blocks: output, per-round counts and
    out-of-order counts (which the carries decide at every bucket boundary) equal the oracle's, and
    the seam repairs equal their definition."""
    rs = np.random.RandomState(77)
    n = 3_000_001  # 7,324 buckets of 2^9 positions: eight tiles of the scans
    # distinct keys: without carried rows, ties between buckets are broken by in-bucket order, so
    # the out-of-order counts equal the oracle's (which breaks them by row) only without ties
    keys = rs.permutation(n).astype(np.float32)
    L, _, _ = orc.nm_split(n)
    rank = keys.astype(np.int64)
    # near-sorted positions with collisions and a few keys moved thousands of positions: several
    # rounds, out-of-order elements and carries across buckets
    slots = (rank * 5 // 4 + rs.randint(-1, 2, n)).astype(np.int64)
    idx = rs.choice(n, 300, replace=False)
    slots[idx] += rs.randint(-3000, 3000, 300)
    slots = np.clip(slots, 0, L - 1).astype(np.uint32)
    dk, kt = to_dev(keys)
    ds = torch.from_numpy(slots.view(np.int32)).cuda()
    st = nns.sort(dk, None, None, eps=3, tau=0, slots=ds, key_type=kt, bucket_log2=9)
    ok, _, ost, _ = orc.nnsort(keys, slots, L, 3, 0)
    np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(ok))
    assert stats_core(st) == stats_core(ost)
    assert st["t"] >= 2 and sum(st["out_of_order"]) > 0
    # seam: keys sent across bucket boundaries, every repair range as defined
    slots2 = (rank * 5 // 4).astype(np.int64)
    idx = rs.choice(n, 2000, replace=False)
    slots2[idx] += rs.randint(-300, 300, 2000)
    slots2 = np.clip(slots2, 0, L - 1).astype(np.uint32)
    dk, kt = to_dev(keys)
    ds = torch.from_numpy(slots2.view(np.int32)).cuda()
    st2 = nns.sort(dk, None, None, slots=ds, key_type=kt, bucket_log2=9)
    np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(np.sort(keys, kind="stable")))
    assert (st2["repair_ranges"], st2["repaired"]) == _expected_seam(keys, slots2, 9)
    assert st2["repair_ranges"] > 0


def test_many_long_seam_ranges_sorted_together():
    """Five stretches of the key order mapped to positions in reverse: five unsound ranges of
    ~180K keys each (longer than one block repairs), separated by sound cuts, repaired by one packed
    multi-block sort. With a payload (and a non-monotone model, so that no row trace is kept) the
    payload follows its keys and equal keys keep input order."""
    n = 2_000_000
    rs = np.random.RandomState(77)
    keys = np.round(W.uniform_f32(n, 22) * 1e5).astype(np.float32)  # many equal keys
    L, _, _ = orc.nm_split(n)
    rank = np.argsort(np.argsort(keys, kind="stable"), kind="stable")
    slots = (rank * 5 // 4).astype(np.int64)
    for c in rs.choice(np.arange(1, 9), 5, replace=False):
        lo, hi = c * 200_000, c * 200_000 + 180_000
        sel = (rank >= lo) & (rank < hi)
        slots[sel] = (lo * 5 // 4) + ((hi - 1 - rank[sel]) * 5 // 4)
    slots = np.clip(slots, 0, L - 1).astype(np.uint32)
    dk, kt = to_dev(keys)
    ds = torch.from_numpy(slots.view(np.int32)).cuda()
    st = nns.sort(dk, None, None, slots=ds, key_type=kt, bucket_log2=12)
    np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(np.sort(keys, kind="stable")))
    cnt, elems = _expected_seam(keys, slots, 12)
    assert (st["repair_ranges"], st["repaired"]) == (cnt, elems)
    assert cnt >= 5 and elems > 5 * 65_536
    # payload through the model path: an untrained two-layer model is non-monotone
    keys = np.round(W.lognormal_f32(1_500_000, 23, sigma=1.0) * 1e3).astype(np.float32)
    payload = np.arange(keys.shape[0], dtype=np.int32)
    om = _rand_model(orc.F32, keys, 2, 16, 16, orc.ORDBITS, seed=9)
    dk, _ = to_dev(keys)
    dp = torch.from_numpy(payload).cuda()
    st = nns.sort(dk, dp, lib_model(om))
    ok, op, ost, _ = orc.nnsort_model(keys, om, payload=payload)
    np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(ok))
    np.testing.assert_array_equal(dp.cpu().numpy(), op)
    assert stats_core(st) == stats_core(ost)
    assert st["repaired"] > 65_536


def test_batch_long_seams_stay_in_their_array():
    """Arrays over the same key range, each with a non-monotone (untrained) model: every array has
    seam ranges longer than one block repairs; they are sorted together by key and then by array,
    so no key moves to another array. Payload rows follow their keys."""
    arrs, oms, pays = [], [], []
    for j in range(7):
        a = W.uniform_f32(200_000 + 37_000 * j, 60 + j)
        arrs.append(a)
        oms.append(_rand_model(orc.F32, a, 2, 16, 16, orc.ORDBITS, seed=20 + j))
        pays.append(np.arange(a.shape[0], dtype=np.int32))
    dks = [to_dev(a)[0] for a in arrs]
    dps = [torch.from_numpy(p.copy()).cuda() for p in pays]
    sts = nns.sort_batch(dks, [lib_model(om) for om in oms], dps)
    for a, om, p, dk, dp, st in zip(arrs, oms, pays, dks, dps, sts):
        ok, op, ost, _ = orc.nnsort_model(a, om, payload=p)
        np.testing.assert_array_equal(bits(from_dev(dk, a)), bits(ok))
        np.testing.assert_array_equal(dp.cpu().numpy(), op)
        assert stats_core(st) == stats_core(ost)
    assert sum(st["repaired"] > 65_536 for st in sts) >= 2


# ---------------------------------------------------------------------------- giant buckets
def test_giant_buckets_sorted_multi_block():
    """Buckets holding more than 65,536 elements are polished by splitting their runs on chip and
    sorting their elements in one multi-block sort: outputs, per-iteration counts and out-of-order
    counts equal the oracle's."""
    rs = np.random.RandomState(31)
    n = 400_000
    keys = W.normal_f32(n, 32)
    L, _, _ = orc.nm_split(n)
    rank = np.argsort(np.argsort(keys, kind="stable"), kind="stable")
    slots = (rank * 5 // 4).astype(np.int64)
    # two crowded stretches: 25% of the keys on 100 positions, 20% on 3000 positions elsewhere
    c1 = rs.rand(n) < 0.25
    slots[c1] = 9000 + (slots[c1] % 100)
    c2 = (~c1) & (rs.rand(n) < 0.27)
    slots[c2] = 300_000 + (slots[c2] % 3000)
    slots = slots.astype(np.uint32)
    for eps in (1, 3):
        dk, kt = to_dev(keys)
        ds = torch.from_numpy(slots.view(np.int32)).cuda()
        st = nns.sort(dk, None, None, slots=ds, eps=eps, tau=0, key_type=kt, bucket_log2=12)
        ok, _, ost, _ = orc.nnsort(keys, slots, L, eps, 0)
        np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(ok))
        assert stats_core(st) == stats_core(ost)
        assert st["oversized_buckets"] >= 2
    # with a payload and the per-row fates (rows are carried: the rounds of giant buckets use rows as
    # the tie-break, their polish stays on one block)
    _check_injected(keys, slots, L, 3, 0, payload=np.arange(n, dtype=np.int32), bucket_log2=12)
    # through a model that sends the lowest 30% of the keys to position 0, with a payload
    keys = W.uniform_f32(500_000, 33)
    payload = np.arange(keys.shape[0], dtype=np.int32)
    nm = orc.make_norm(keys, np.arange(keys.shape[0], dtype=np.uint64), orc.VALUE)
    p = np.zeros(3 * 8 + 1, np.float32)
    p[0], p[8], p[16] = 1.0, -0.3, 1.0 / 0.7  # F(x) = relu(x - 0.3) / 0.7
    om = orc.Model(1, 8, 0, nm, p)
    dk, _ = to_dev(keys)
    dp = torch.from_numpy(payload.copy()).cuda()
    st = nns.sort(dk, dp, lib_model(om))
    ok, op, ost, _ = orc.nnsort_model(keys, om, payload=payload)
    np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(ok))
    np.testing.assert_array_equal(dp.cpu().numpy(), op)
    assert stats_core(st) == stats_core(ost)
    assert st["oversized_buckets"] >= 1


# ---------------------------------------------------------------------------- no-model reference
def test_radix_sort_reference_is_the_stable_sort():
    """nnsort_radix_sort (the ablation's "no model" reference: every pass the partition kernel on
    8-bit key digits) gives the stable order by (key, row): keys bit-exact, payload = stable
    permutation, for f32 (signed zeros, infinities, duplicates, a ragged tail), f64 and u64."""
    rs = np.random.RandomState(77)
    f = W.lognormal_dup_f32(300_001, 5, sigma=2.0)
    f[:6] = [-0.0, 0.0, np.inf, -np.inf, -1.5, 0.0]
    cases = [f, rs.standard_normal(123_457), (rs.randint(0, 2 ** 63, 200_003, dtype=np.int64)
                                              .astype(np.uint64) * np.uint64(2))]
    for keys in cases:
        payload = np.arange(keys.shape[0], dtype=np.int32)
        dk, kt = to_dev(keys)
        dp = torch.from_numpy(payload).cuda()
        nns.radix_sort(dk, dp, key_type=kt)
        ok, op = orc.stable_sort(keys, payload)
        np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(ok))
        np.testing.assert_array_equal(dp.cpu().numpy(), op)
        dk, kt = to_dev(keys)
        nns.radix_sort(dk, None, key_type=kt)  # keys only
        np.testing.assert_array_equal(bits(from_dev(dk, keys)), bits(ok))
    nns.radix_sort(torch.empty(0, device="cuda"))
