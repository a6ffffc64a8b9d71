"""nnsort_sort_noalloc: the sort for callers that cannot allocate device memory when they sort
(a memory budget fixed up front, no cudaMalloc/cudaFree on the critical path, or an allocator owned
by another framework). It takes its scratch from the library's fixed device array instead of
allocating, and must give the same result as nnsort_sort. Called through the C ABI, twice in a row,
so the second call runs on scratch the first call left behind."""
import ctypes as C

import numpy as np
import pytest

from helpers import lib_model
from oracle import oracle as orc
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)
import paper_1907_08817_gb300 as nns  # noqa: E402
from paper_1907_08817_gb300 import _lib as L  # noqa: E402


def _noalloc(keys, payload, dtype_code, model, m=1.25, precision="fp32", bucket_log2=0):
    o = nns._sopts(m, 3, 1024, precision, bucket_log2, None, None, False)
    st = L.Stats()
    rc = L.lib().nnsort_sort_noalloc(
        C.c_void_p(keys.data_ptr()), None if payload is None else C.c_void_p(payload.data_ptr()),
        keys.numel(), dtype_code, model.handle, C.byref(o), C.byref(st),
        C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, st.as_dict()


def _case(seed, n, kv, u64):
    if u64:
        keys, _ = W.gauss_mix_u64(n, seed)
        om, _, _ = orc.train(keys, 2, 16, 16, orc.ORDBITS, sample_n=2000, steps=40, seed=seed)
        dev = torch.from_numpy(keys.view(np.int64)).cuda()
        code = 3
    else:
        keys = W.lognormal_dup_f32(n, seed, sigma=2.0)
        om, _, _ = orc.train(keys, 1, 32, 0, orc.ORDBITS, sample_n=2000, steps=50, seed=seed)
        dev = torch.from_numpy(keys).cuda()
        code = 0
    payload = torch.arange(n, dtype=torch.int32, device="cuda") if kv else None
    return dev, payload, code, lib_model(om)


def test_noalloc_matches_nnsort_sort_on_two_calls_in_a_row():
    cases = [(21, 200_000, True, False), (22, 262_144, False, True)]
    for seed, n, kv, u64 in cases:
        dev, payload, code, f = _case(seed, n, kv, u64)
        a, b = dev.clone(), dev.clone()
        pa = None if payload is None else payload.clone()
        pb = None if payload is None else payload.clone()
        ref = nns.sort(a, pa, f, key_type="u64" if u64 else None)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        rc, st = _noalloc(b, pb, code, f)
        free1, _ = torch.cuda.mem_get_info()
        assert rc == 0, L.STATUS.get(rc, rc)
        # same stable order as the allocating entry point, bit for bit
        assert torch.equal(a.view(torch.int32), b.view(torch.int32))
        if pa is not None:
            assert torch.equal(pa, pb)
        for k in ("t", "w_size", "placed", "out_of_order"):
            assert st[k] == ref[k]
        # after the first call on the device nothing further is allocated
        if seed == 22:
            assert free1 == free0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    n = 262_145  # NNSORT_NOALLOC_MAX_N + 1
    keys = torch.rand(n, device="cuda")
    om = orc.Model(1, 8, 0, orc.make_norm(keys[:100].cpu().numpy(), np.arange(100, dtype=np.uint64),
                                         orc.VALUE), orc.init_params(1, 8, 0, 0))
    before = keys.clone()
    rc, _ = _noalloc(keys, None, 0, lib_model(om))
    assert rc == -1
    assert torch.equal(before, keys)


def _expect(dev, payload, code):
    """The stable order from the oracle's library sort of the same keys (and payload)."""
    like = {0: np.float32, 3: np.uint64}[code]
    keys = dev.cpu().numpy().view(like)
    pay = None if payload is None else payload.cpu().numpy()
    return orc.stable_sort(keys, pay)


def test_noalloc_tensor_core_form_matches_nnsort_sort():
    """Split BF16 inference of a 1-64-64-1 model: the single-array tensor-core kernel, as in
    nnsort_sort; keys, payload and the per-round statistics agree."""
    n = 250_000
    keys = W.lognormal_dup_f32(n, 31, sigma=2.0)
    om, _, _ = orc.train(keys, 2, 64, 64, orc.ORDBITS, sample_n=2000, steps=30, seed=31)
    f = lib_model(om)
    for prec in ("bf16x2", "bf16"):
        dev = torch.from_numpy(keys).cuda()
        pay = torch.arange(n, dtype=torch.int32, device="cuda")
        a, b, pa, pb = dev.clone(), dev.clone(), pay.clone(), pay.clone()
        ref = nns.sort(a, pa, f, precision=prec, bucket_log2=12, eps=3)
        rc, st = _noalloc(b, pb, 0, f, precision=prec, bucket_log2=12)
        assert rc == 0, L.STATUS.get(rc, rc)
        assert torch.equal(a.view(torch.int32), b.view(torch.int32))
        assert torch.equal(pa, pb)
        for k in ("t", "w_size", "placed", "out_of_order"):
            assert st[k] == ref[k], (prec, k)


def test_noalloc_one_bucket_two_passes_and_repeated_calls():
    """(1) Nearly all keys equal, so one bucket holds ~99% of the 262,144 keys (the one-block
    rounds and sort over global lists); (2) 512-position buckets with m = 1.9, so 973 buckets need
    two partition passes; run four times in a row, each call on the scratch the previous one
    left. Each result equals the oracle's stable sort and nnsort_sort's statistics."""
    n = 262_144
    rs = np.random.RandomState(41)
    dup = np.full(n, 3.5, np.float32)
    odd = rs.rand(n) < 0.01
    dup[odd] = W.lognormal_f32(int(odd.sum()), 41, 0.0, 2.0)
    spread = W.lognormal_dup_f32(n, 42, sigma=2.0)
    cases = []
    for keys, m, wlog in ((dup, 1.25, 12), (spread, 1.9, 9)):
        om, _, _ = orc.train(keys, 1, 32, 0, orc.ORDBITS, sample_n=2000, steps=50, seed=5)
        cases.append((keys, m, wlog, lib_model(om)))
    for rep in range(2):
        for keys, m, wlog, f in cases:
            dev = torch.from_numpy(keys).cuda()
            pay = torch.arange(n, dtype=torch.int32, device="cuda")
            ek, ep = _expect(dev, pay, 0)
            a, pa = dev.clone(), pay.clone()
            ref = nns.sort(a, pa, f, m=m, bucket_log2=wlog, eps=3)
            rc, st = _noalloc(dev, pay, 0, f, m=m, bucket_log2=wlog)
            assert rc == 0, L.STATUS.get(rc, rc)
            assert np.array_equal(dev.cpu().numpy().view(np.uint32), ek.view(np.uint32))
            assert np.array_equal(pay.cpu().numpy(), ep)
            for k in ("t", "w_size", "placed", "out_of_order"):
                assert st[k] == ref[k], (m, wlog, k)
            if wlog == 9:
                assert ref["partition_passes"] == 2
            else:
                assert max(st["w_size"][1:] or [0]) > 0


def test_noalloc_rejects_position_counts_beyond_its_bucket_tables():
    """A relaxation factor whose position count n m exceeds the fixed bucket tables (or is not
    finite) is rejected before any narrowing, with the keys left as they were."""
    n = 1000
    keys = torch.rand(n, device="cuda")
    om = orc.Model(1, 8, 0, orc.make_norm(keys[:100].cpu().numpy(), np.arange(100, dtype=np.uint64),
                                         orc.VALUE), orc.init_params(1, 8, 0, 0))
    f = lib_model(om)
    before = keys.clone()
    for m in (1e30, float("inf"), 5000.0):
        rc, _ = _noalloc(keys, None, 0, f, m=m)
        assert rc == -1, m
        assert torch.equal(before, keys)
