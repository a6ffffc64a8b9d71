"""Seeded synthetic inputs for NN-sort: the key arrays every test and the benchmark feed to both
the CUDA path and the oracle.

This module draws random numbers and shapes them into workloads. It holds none of the sorting
method's arithmetic (no translation, no model, no slot or ordering logic), so the oracle and the
CUDA path can both be fed from it without sharing any code of the method.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used as a counter-based generator: the i-th draw of stream `seed` is the
SplitMix64 output function applied to `seed + (i + 1) * 0x9E3779B97F4A7C15`.

Workloads (the paper's Experimental Study uses uniform, normal and lognormal 64-bit floats of
200-500 MB; the sizes and distributions below are the synthetic stand-ins this project measures):

- ``uniform_f32``      n float32 keys U[0,1) with 24 random mantissa bits.
- ``lognormal_dup_f32`` n float32 keys; 95% draws exp(mu + sigma N(0,1)), 5% exact copies of
  uniformly chosen base draws, then shuffled.
- ``gauss_mix_u64``    n uint64 keys from a mixture of 8 Gaussians with Zipf(s=1.1) weights and means
  spread over [0, 2^63), low 11 bits uniform; payload = original index.
- ``batch_arrays``     many float32 arrays of log-uniform sizes, each from one of
  uniform / normal / lognormal / exponential.
- ``serving_requests`` float64 request arrays of log-uniform sizes from mixed distributions with
  Poisson arrival times.
- ``shift_mix_f32``    uniform float32 keys with a share replaced by normal "noise" (Exp-3).
- ``uniform_u64``      uint64 keys uniform over the full range (the QuickDraw-sized stand-in, Exp-2).
"""
from __future__ import annotations

import concurrent.futures as cf
import os

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22


def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def rng_u64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws start .. start+count-1 of the SplitMix64 stream `seed` (uint64)."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * GAMMA)


def stream_seed(seed: int, tag: int) -> int:
    """Independent sub-stream for one purpose (tag) of a workload seed."""
    return int(rng_u64(seed, tag, 1)[0])


def _unit_f64(u: np.ndarray) -> np.ndarray:
    """uint64 -> double in [0, 1) from the top 53 bits."""
    return (u >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _normal_f64(seed: int, start: int, count: int) -> np.ndarray:
    """Box-Muller standard normals; draw k uses stream draws 2k and 2k+1."""
    u = rng_u64(seed, 2 * start, 2 * count)
    u1 = ((u[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)
    u2 = _unit_f64(u[1::2])
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def _chunked(n: int, fn, dtype) -> np.ndarray:
    """fn(start, count) for consecutive chunks of [0, n); chunks are independent (counter-based
    draws), so they are computed on a thread pool (numpy releases the GIL) with the same result."""
    out = np.empty(n, dtype=dtype)

    def one(s):
        c = min(_CHUNK, n - s)
        out[s:s + c] = fn(s, c)
    starts = range(0, n, _CHUNK)
    if n <= _CHUNK or _threads() == 1:
        for s in starts:
            one(s)
    else:
        with cf.ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(one, starts))
    return out


def uniform_f32(n: int, seed: int = 0) -> np.ndarray:
    """float32 keys U[0,1): (u >> 40) * 2^-24 (24 random bits)."""
    return _chunked(n, lambda s, c: ((rng_u64(seed, s, c) >> np.uint64(40)).astype(np.float64)
                                     * (1.0 / 16777216.0)).astype(np.float32), np.float32)


def normal_f32(n: int, seed: int = 0, mu: float = 0.0, sigma: float = 1.0) -> np.ndarray:
    return _chunked(n, lambda s, c: (mu + sigma * _normal_f64(seed, s, c)).astype(np.float32),
                    np.float32)


def lognormal_f32(n: int, seed: int = 0, mu: float = 0.0, sigma: float = 1.0) -> np.ndarray:
    return _chunked(n, lambda s, c: np.exp(mu + sigma * _normal_f64(seed, s, c)).astype(np.float32),
                    np.float32)


def exponential_f32(n: int, seed: int = 0, lam: float = 1.0) -> np.ndarray:
    def f(s, c):
        u = _unit_f64(rng_u64(seed, s, c))
        return (-np.log1p(-u) / lam).astype(np.float32)
    return _chunked(n, f, np.float32)


def _permute_inplace(a: np.ndarray, seed: int) -> np.ndarray:
    perm = np.random.Generator(np.random.PCG64(seed)).permutation(a.shape[0])
    return a[perm]


def lognormal_dup_f32(n: int, seed: int = 2, mu: float = 0.0, sigma: float = 2.0,
                      dup_frac: float = 0.05) -> np.ndarray:
    """float32 lognormal(mu, sigma) keys with `dup_frac` exact duplicates of earlier draws, shuffled."""
    n_dup = int(round(n * dup_frac))
    n_base = n - n_dup
    keys = np.empty(n, dtype=np.float32)
    keys[:n_base] = lognormal_f32(n_base, stream_seed(seed, 1), mu, sigma)
    if n_dup:
        s2 = stream_seed(seed, 2)
        src = _chunked(n_dup, lambda s, c: _mulhi(rng_u64(s2, s, c), n_base), np.int64)
        keys[n_base:] = keys[src]
    return _permute_inplace(keys, seed)


def _mulhi(u: np.ndarray, n: int) -> np.ndarray:
    """floor(u * n / 2^64) for uint64 u and n < 2^32 (uniform index in [0, n))."""
    assert 0 < n < (1 << 32)
    lo = u & np.uint64(0xFFFFFFFF)
    hi = u >> np.uint64(32)
    nn = np.uint64(n)
    t = (lo * nn) >> np.uint64(32)
    return ((hi * nn + t) >> np.uint64(32)).astype(np.int64)


def gauss_mix_u64(n: int, seed: int = 3, components: int = 8, zipf_s: float = 1.1):
    """uint64 keys from a mixture of Gaussians; returns (keys, payload) with payload = index (int32)."""
    w = np.arange(1, components + 1, dtype=np.float64) ** (-zipf_s)
    cdf = np.cumsum(w / w.sum())
    two63 = float(2 ** 63)
    mus = (2.0 * np.arange(1, components + 1) - 1.0) / (2.0 * components) * two63
    sd = two63 / 64.0

    def f(s, c):
        comp = np.searchsorted(cdf, _unit_f64(rng_u64(stream_seed(seed, 1), s, c)), side="right")
        comp = np.minimum(comp, components - 1)
        v = mus[comp] + sd * _normal_f64(stream_seed(seed, 2), s, c)
        v = np.clip(np.rint(v), 0.0, 18446744073709549568.0)
        k = v.astype(np.uint64)
        low = rng_u64(stream_seed(seed, 3), s, c) & np.uint64(0x7FF)
        return (k & ~np.uint64(0x7FF)) | low
    keys = _chunked(n, f, np.uint64)
    payload = np.arange(n, dtype=np.int32)
    return keys, payload


_DISTS = ("uniform", "normal", "lognormal", "exponential")


def dist_f32(kind: str, n: int, seed: int) -> np.ndarray:
    if kind == "uniform":
        return uniform_f32(n, seed)
    if kind == "normal":
        return normal_f32(n, seed)
    if kind == "lognormal":
        return lognormal_f32(n, seed)
    if kind == "exponential":
        return exponential_f32(n, seed)
    raise ValueError(kind)


def batch_arrays(count: int = 4096, seed: int = 4, lo: int = 1000, hi: int = 1_000_000,
                 total_cap: int | None = None):
    """List of (kind, float32 array) with sizes floor(lo * (hi/lo)^U), kind uniform over four
    distributions. `total_cap` truncates the list once the running total would exceed it."""
    u = _unit_f64(rng_u64(stream_seed(seed, 1), 0, count))
    sizes = np.floor(lo * (hi / lo) ** u).astype(np.int64)
    kinds = (rng_u64(stream_seed(seed, 2), 0, count) % np.uint64(len(_DISTS))).astype(np.int64)
    take = count
    if total_cap is not None:
        csum = np.cumsum(sizes)
        take = int(np.searchsorted(csum, total_cap, side="right"))

    def one(j):
        return (_DISTS[kinds[j]], dist_f32(_DISTS[kinds[j]], int(sizes[j]), stream_seed(seed, 100 + j)))
    if take > 8 and _threads() > 1:
        with cf.ThreadPoolExecutor(_threads()) as ex:
            return list(ex.map(one, range(take)))
    return [one(j) for j in range(take)]


def serving_requests(count: int = 1000, seed: int = 5, lo: int = 10_000, hi: int = 16_000_000,
                     rate_per_s: float = 100.0, max_keys: int | None = None):
    """List of dicts {arrival_s, kind, keys(float64)}: sizes log-uniform in [lo, hi], kinds
    uniform / lognormal(0,2) / clustered (16 centres U[0,1e6) with N(0,1) spread), Poisson arrivals
    at `rate_per_s`."""
    u = _unit_f64(rng_u64(stream_seed(seed, 1), 0, count))
    sizes = np.floor(lo * (hi / lo) ** u).astype(np.int64)
    if max_keys is not None:
        sizes = np.minimum(sizes, max_keys)
    kinds = (rng_u64(stream_seed(seed, 2), 0, count) % np.uint64(3)).astype(np.int64)
    gaps = -np.log1p(-_unit_f64(rng_u64(stream_seed(seed, 3), 0, count))) / rate_per_s
    arrivals = np.cumsum(gaps)
    def one(j):
        n = int(sizes[j])
        s = stream_seed(seed, 1000 + j)
        if kinds[j] == 0:
            keys = _unit_f64(rng_u64(s, 0, n))
            kind = "uniform"
        elif kinds[j] == 1:
            keys = np.exp(2.0 * _normal_f64(s, 0, n))
            kind = "lognormal"
        else:
            centres = _unit_f64(rng_u64(stream_seed(s, 7), 0, 16)) * 1e6
            which = (rng_u64(stream_seed(s, 8), 0, n) % np.uint64(16)).astype(np.int64)
            keys = centres[which] + _normal_f64(stream_seed(s, 9), 0, n)
            kind = "clustered"
        return {"arrival_s": float(arrivals[j]), "kind": kind, "keys": keys.astype(np.float64)}
    if count > 8 and _threads() > 1:
        with cf.ThreadPoolExecutor(_threads()) as ex:
            return list(ex.map(one, range(count)))
    return [one(j) for j in range(count)]


def shift_mix_f32(n: int, noise_frac: float, seed: int = 6, mu: float = 0.5,
                  sigma: float = 0.1) -> np.ndarray:
    """float32 keys for the changing-distribution experiment (Exp-3): U[0,1) draws with a share
    `noise_frac` replaced by normal(mu, sigma) draws (the "noise"), shuffled. The paper does not
    state the normal's parameters; N(0.5, 0.1) keeps the noise inside the uniform range, so it
    crowds keys into the middle instead of widening the range."""
    n_noise = int(round(n * noise_frac))
    keys = np.empty(n, dtype=np.float32)
    keys[:n - n_noise] = uniform_f32(n - n_noise, stream_seed(seed, 1))
    if n_noise:
        keys[n - n_noise:] = normal_f32(n_noise, stream_seed(seed, 2), mu, sigma)
    return _permute_inplace(keys, seed)


QUICKDRAW_RECORDS = 50_426_265


def uniform_u64(n: int, seed: int = 7) -> np.ndarray:
    """uint64 keys uniform over [0, 2^64): the stand-in for the QuickDraw key-ids (Exp-2), whose
    records are not available here; QUICKDRAW_RECORDS is the dataset's size."""
    return _chunked(n, lambda s, c: rng_u64(seed, s, c), np.uint64)
