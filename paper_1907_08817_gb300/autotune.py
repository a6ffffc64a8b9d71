"""Autotuner for the sort's tile and round parameters.

Searches, for one class of workload, the bucket width (positions per on-chip bucket, 2^9..2^14),
the number of polish blocks per SM (on-chip capacity against overlap) and the round limit eps, by
timing the sort (CUDA events recorded inside the library) on a representative input with its
trained model; the output is identical for every candidate, only time and statistics change. The
result is stored in a JSON table keyed by (key type, log2 n, model shape, precision) and looked up
by `tuned_options`, which `sort`/`sort_batch` callers can splat into their keyword arguments.

The table shipped in this package (tuned.json) is written by `python -m
paper_1907_08817_gb300.autotune --write [--out PATH]` on the target GPU.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import statistics
from typing import Callable, Iterable

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuned.json")

DEFAULT_SPACE = {
    "bucket_log2": (10, 11, 12, 13),
    "polish_blocks": (1, 2, 3),
    "eps": (1, 2, 3, 4),
}
DEFAULTS = {"bucket_log2": 12, "polish_blocks": 3, "eps": 3}


def table_key(dtype: int, n: int, layers: int, h1: int, h2: int, precision: str) -> str:
    return f"d{dtype}-n{max(0, int(math.log2(max(n, 1))))}-l{layers}-{h1}x{h2}-{precision}"


def search(measure: Callable[[dict], float], space: dict | None = None, repeats: int = 3,
           coordinate: bool = True) -> tuple[dict, list]:
    """Minimises measure(config) (a time) over the space. With coordinate=True each parameter is
    optimised in turn starting from DEFAULTS (two sweeps), otherwise the full grid is timed.
    Returns (best config, [(config, median time), ...])."""
    space = space or DEFAULT_SPACE
    cache: dict = {}

    def timed(cfg: dict) -> float:
        k = tuple(sorted(cfg.items()))
        if k not in cache:
            cache[k] = statistics.median(measure(dict(cfg)) for _ in range(repeats))
        return cache[k]

    if not coordinate:
        names = list(space)
        best = None
        for vals in itertools.product(*(space[n] for n in names)):
            cfg = dict(zip(names, vals))
            if best is None or timed(cfg) < timed(best):
                best = cfg
    else:
        best = {k: DEFAULTS.get(k, v[0]) for k, v in space.items()}
        for _ in range(2):
            for name, values in space.items():
                for v in values:
                    cfg = dict(best, **{name: v})
                    if timed(cfg) < timed(best):
                        best = cfg
    log = [(dict(k), t) for k, t in cache.items()]
    return best, log


_cache: dict = {}


def load_table(path: str = TABLE) -> dict:
    """The table at `path` ({} if absent or unreadable), re-read only when the file changes."""
    try:
        mt = os.stat(path).st_mtime_ns
    except OSError:
        return {}
    hit = _cache.get(path)
    if hit is not None and hit[0] == mt:
        return hit[1]
    try:
        with open(path) as f:
            t = json.load(f)
    except (OSError, ValueError):
        t = {}
    _cache[path] = (mt, t)
    return t


def save_entry(key: str, cfg: dict, ms: float, path: str = TABLE) -> None:
    t = dict(load_table(path))
    t[key] = {**cfg, "sort_ms": round(ms, 3)}
    with open(path, "w") as f:
        json.dump(t, f, indent=1, sort_keys=True)
        f.write("\n")
    _cache.pop(path, None)


def tuned_entry(dtype: int, n: int, layers: int, h1: int, h2: int, precision: str,
                path: str = TABLE) -> dict | None:
    """The table entry for this workload class: n's size class, else the nearest tuned size class
    of the same key type, model shape and precision, else None."""
    t = load_table(path)
    key = table_key(dtype, n, layers, h1, h2, precision)
    if key in t:
        return t[key]
    prefix = f"d{dtype}-"
    suffix = key.split("-", 2)[2]
    cands = [(abs(int(k.split("-")[1][1:]) - int(math.log2(max(n, 1)))), k) for k in t
             if k.startswith(prefix) and k.split("-", 2)[2] == suffix]
    return t[min(cands)[1]] if cands else None


PRECISIONS = ("fp32", "bf16x2", "bf16", "pwl")


def tuned_options(dtype: int, n: int, layers: int, h1: int, h2: int, precision: str,
                  path: str = TABLE) -> dict:
    """Tuned keyword arguments for sort()/sort_batch(): the nearest table entry of the same key
    type, model shape and precision; when that precision was never tuned for the class, the entry
    of another precision of the same key type and model shape (bucket width, polish blocks and
    round limit depend on the data and the model far more than on the form of the forward pass);
    else the library defaults."""
    e = tuned_entry(dtype, n, layers, h1, h2, precision, path)
    for other in PRECISIONS:
        if e is not None:
            break
        if other != precision:
            e = tuned_entry(dtype, n, layers, h1, h2, other, path)
    if e is None:
        return dict(DEFAULTS)
    return {k: e[k] for k in DEFAULTS if k in e}


def _event_ms(run) -> float:
    import torch
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(s)
    run()
    b.record(s)
    torch.cuda.synchronize()
    return a.elapsed_time(b)


def tune_gpu(keys_list, models, precision: str, payloads=None, space: dict | None = None,
             repeats: int = 3, write: bool = False, path: str = TABLE, key_type=None):
    """Times the sort of copies of the device tensors in keys_list (one array: nnsort_sort, with the
    library's per-stage times kept in tune_gpu.stages; several: one nnsort_sort_batch) over the
    space; every candidate's output is checked to equal the first's. Returns (best, log) and, with write=True, stores the best under the class of the
    mean array size, the key type and the first model's shape."""
    import torch

    from . import key_code, sort, sort_batch
    work = [k.clone() for k in keys_list]
    wpay = None if payloads is None else [p.clone() for p in payloads]
    first = []
    stages: dict = {}

    def measure(cfg: dict) -> float:
        for w, k in zip(work, keys_list):
            w.copy_(k)
        if wpay is not None:
            for w, p in zip(wpay, payloads):
                w.copy_(p)
        if len(work) == 1:
            def run():
                st = sort(work[0], None if wpay is None else wpay[0], models[0], precision=precision,
                          timing=True, key_type=key_type, **cfg)
                stages[tuple(sorted(cfg.items()))] = [round(v, 3) for v in st["ms_stage"][:7]]
        else:
            run = lambda: sort_batch(work, models, wpay, precision=precision,  # noqa: E731
                                     stats=False, key_type=key_type, **cfg)
        ms = _event_ms(run)
        if not first:
            first.extend(w.clone() for w in work)
        elif not all(torch.equal(a, b) for a, b in zip(first, work)):
            raise RuntimeError(f"autotune: output differs under {cfg}")
        return ms

    best, log = search(measure, space, repeats)
    ms = min(t for c, t in log if c == best)
    tune_gpu.stages = {str(dict(k)): v for k, v in stages.items()}
    if write:
        n = sum(k.numel() for k in keys_list) // len(keys_list)
        save_entry(table_key(key_code(keys_list[0], key_type), n, *models[0].shape, precision),
                   best, ms, path)
    return best, log


def _main(argv: Iterable[str]) -> None:
    import sys

    import numpy as np
    import torch

    sys.path.insert(0, os.path.dirname(HERE))
    import workloads as W

    from . import train
    argv = list(argv)
    write = "--write" in argv
    path = argv[argv.index("--out") + 1] if "--out" in argv else TABLE

    def one(gen, n, arch, steps=100):
        def make():
            k = gen(n)
            pay = None
            if isinstance(k, tuple):
                k, pay = k
            kt = "u64" if k.dtype == np.uint64 else None
            dk = torch.from_numpy(k.view(np.int64) if kt else k).cuda()
            m, _ = train(dk, key_type=kt, layers=arch[0], h1=arch[1], h2=arch[2],
                         sample_n=min(n, 1 << 20) if kt else max(1000, n // 100), steps=steps,
                         batch=65536 if n > (1 << 22) else 0, seed=0)
            return [dk], [m], (None if pay is None else [torch.from_numpy(pay).cuda()]), kt
        return make

    def batch():
        ks, ms = [], []
        for _, a in W.batch_arrays(4096, seed=4, total_cap=200_000_000):
            dk = torch.from_numpy(a).cuda()
            m, _ = train(dk, layers=1, h1=16, h2=0, sample_n=max(100, a.shape[0] // 100), steps=100,
                         batch=0, seed=0)
            ks.append(dk)
            ms.append(m)
        return ks, ms, None, None

    big = one(lambda n: W.lognormal_dup_f32(n, 2, sigma=2.0), 1 << 28, (2, 64, 64))
    c3 = one(lambda n: W.gauss_mix_u64(n, 3), 1 << 26, (2, 32, 32), steps=200)
    cases = [
        # (label, maker, precision); consecutive cases with the same label share the input
        ("lognormal_dup_f32 256M 1-64-64-1", big, "bf16x2"),
        ("lognormal_dup_f32 256M 1-64-64-1", big, "bf16"),
        ("lognormal_dup_f32 256M 1-64-64-1", big, "fp32"),
        ("lognormal_dup_f32 256M 1-64-64-1", big, "pwl"),
        ("uniform_f32 1M 1-32-1", one(lambda n: W.uniform_f32(n, 0), 1_000_000, (1, 32, 0)), "fp32"),
        ("gauss_mix_u64 64M + payload 1-32-32-1", c3, "bf16x2"),
        ("gauss_mix_u64 64M + payload 1-32-32-1", c3, "fp32"),
        ("gauss_mix_u64 64M + payload 1-32-32-1", c3, "pwl"),
        ("batch of f32 arrays 1K..1M 1-16-1", batch, "fp32"),
    ]
    only = argv[argv.index("--case") + 1] if "--case" in argv else None
    made = None
    for ci, (label, make, prec) in enumerate(cases):
        if only is not None and str(ci) not in only.split(","):
            continue
        if made is None or made[0] is not make:
            made = None
            torch.cuda.empty_cache()
            made = (make, make())
        ks, ms, pay, kt = made[1]
        best, log = tune_gpu(ks, ms, prec, pay, write=write, path=path, key_type=kt)
        print(json.dumps({"case": label, "arrays": len(ks), "precision": prec, "best": best,
                          "ms": min(t for c, t in log if c == best),
                          "default_ms": next((t for c, t in log if c == DEFAULTS), None),
                          "log": log, "stage_ms": getattr(tune_gpu, "stages", {})}), flush=True)
        del ks, ms, pay


if __name__ == "__main__":
    import sys
    _main(sys.argv[1:])
