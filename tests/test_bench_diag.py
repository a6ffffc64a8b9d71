"""Host-side checks of bench.py's split-BF16 displacement diagnostic (no GPU)."""
import importlib.util
import os
import sys

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    argv = sys.argv
    try:
        sys.argv = ["bench.py"]
        spec.loader.exec_module(mod)
    finally:
        sys.argv = argv
    return mod


def test_bf16_rounding_matches_torch():
    b = _bench()
    rs = np.random.RandomState(3)
    x = np.concatenate([rs.randn(4096).astype(np.float32) * 10.0 ** rs.randint(-8, 8, 4096),
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -1.5, 0.0, 65504.0],
                                 dtype=np.float32)])
    want = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(b._bf16_rn(x), want)


def test_w2_split_displacement_orders_the_three_forms():
    b = _bench()
    rs = np.random.RandomState(0)
    h1 = h2 = 64
    params = (rs.randn(2 * h1 + h2 * h1 + 2 * h2 + 1) * 0.3).astype(np.float32)
    keys = np.exp(rs.randn(1 << 14) * 2).astype(np.float32)
    u = keys.view(np.uint32).astype(np.uint64) | 0x80000000
    desc = {"layers": 2, "h1": h1, "h2": h2, "lo_bits": int(u.min()),
            "scale": 1.0 / float(u.max() - u.min())}
    out = b.w2_split_displacement(keys, desc, params, (1 << 28) * 1.25)
    kern = out["as the kernel (W2 in BF16 for the BF16 part, FP16 for the rest)"]["mean_abs"]
    hilo = out["W2 carried as BF16 part + BF16 rest"]["mean_abs"]
    exact = out["exact W2 (activations split only)"]["mean_abs"]
    assert out["sample_keys"] == keys.size
    # W2 rounded to 8 significant bits dominates; its BF16 rest removes most of it
    assert exact <= hilo < kern
    assert kern > 100 * hilo
