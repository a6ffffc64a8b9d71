"""The seeded input generators (host only, no GPU): each follows the recipe the benchmark and the
tests state for it — counter-based SplitMix64 draws (checked against the generator's published
output), deterministic per seed, and the shapes, ranges and mixtures of the paper's workloads."""
import numpy as np

import workloads as W


def test_splitmix64_reference_outputs():
    # the first outputs of SplitMix64 seeded with 0 (Steele, Lea & Flood; the widely published
    # test vector of the reference implementation)
    want = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    got = [int(v) for v in W.rng_u64(0, 0, 3)]
    assert got == want
    # counter-based: any window of the stream equals the matching slice of a longer draw
    np.testing.assert_array_equal(W.rng_u64(7, 5, 10), W.rng_u64(7, 0, 15)[5:])


def test_generators_are_deterministic_per_seed():
    for gen in (W.uniform_f32, W.normal_f32, W.lognormal_f32, W.exponential_f32):
        a, b, c = gen(10_000, 3), gen(10_000, 3), gen(10_000, 4)
        np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
        assert not np.array_equal(a, c)
    np.testing.assert_array_equal(W.uniform_u64(1000, 1), W.uniform_u64(1000, 1))


def test_uniform_f32_has_24_random_bits_in_unit_interval():
    k = W.uniform_f32(200_000, 0)
    assert k.dtype == np.float32 and k.min() >= 0.0 and k.max() < 1.0
    np.testing.assert_array_equal(k.astype(np.float64) * 2 ** 24, np.floor(k.astype(np.float64) * 2 ** 24))
    assert abs(k.mean() - 0.5) < 0.005


def test_lognormal_dup_share_and_distribution():
    n = 200_000
    k = W.lognormal_dup_f32(n, 2, sigma=2.0, dup_frac=0.05)
    # every duplicate copies an earlier base draw: at least 5% of the keys repeat a value
    _, counts = np.unique(k, return_counts=True)
    assert n - counts.size >= int(0.05 * n) * 0.98
    # log of the base draws is N(0, 2)
    lk = np.log(k.astype(np.float64))
    assert abs(lk.mean()) < 0.05 and abs(lk.std() - 2.0) < 0.05


def test_shift_mix_noise_share():
    n = 200_000
    clean = W.shift_mix_f32(n, 0.0, seed=6)
    assert clean.min() >= 0.0 and clean.max() < 1.0 and abs(clean.std() - np.sqrt(1 / 12)) < 0.003
    pure = W.shift_mix_f32(n, 1.0, seed=6)
    assert abs(pure.mean() - 0.5) < 0.002 and abs(pure.std() - 0.1) < 0.002
    # with a share x of noise, the fraction of keys within 0.05 of 0.5 grows from 0.1 towards 0.38
    for x in (0.15, 0.45):
        mix = W.shift_mix_f32(n, x, seed=6)
        near = np.mean(np.abs(mix - 0.5) < 0.05)
        want = (1 - x) * 0.1 + x * 0.3829
        assert abs(near - want) < 0.01, (x, near, want)


def test_uniform_u64_covers_the_full_range():
    k = W.uniform_u64(100_000, 7)
    assert k.dtype == np.uint64
    top = (k >> np.uint64(56)).astype(np.int64)
    counts = np.bincount(top, minlength=256)
    expected = k.size / 256
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert chi2 < 400  # 255 degrees of freedom
    assert W.QUICKDRAW_RECORDS == 50_426_265


def test_gauss_mix_payload_is_the_index_and_keys_are_clustered():
    k, p = W.gauss_mix_u64(100_000, 3)
    np.testing.assert_array_equal(p, np.arange(100_000, dtype=np.int32))
    assert k.max() < np.uint64(1 << 63) + np.uint64(1 << 61)
    # Zipf(1.1) weights: the first component (mean 2^63 / 16) holds the largest share
    comp = np.floor(k.astype(np.float64) / 2.0 ** 63 * 8).astype(np.int64)
    counts = np.bincount(np.clip(comp, 0, 7), minlength=8)
    assert counts[0] == counts.max()


def test_batch_sizes_are_log_uniform_in_range():
    arrs = W.batch_arrays(64, seed=4, lo=1000, hi=1_000_000)
    sizes = np.array([a.shape[0] for _, a in arrs])
    assert len(arrs) == 64 and sizes.min() >= 1000 and sizes.max() <= 1_000_000
    kinds = {k for k, _ in arrs}
    assert kinds <= {"uniform", "normal", "lognormal", "exponential"} and len(kinds) >= 3
    capped = W.batch_arrays(64, seed=4, total_cap=2_000_000)
    assert sum(a.shape[0] for _, a in capped) <= 2_000_000
