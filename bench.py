#!/usr/bin/env python
"""Benchmark: NN-sort on one GB300 (or N independent replicas under torchrun).

Headline workload (the large single-GPU configuration): 268,435,456 float32 keys, lognormal(0, 2)
with 5% exact duplicates, shuffled, keys only; model f = MLP 1 -> 64 -> 64 -> 1 trained on the
device (1% sample, 100 Adam steps, mini-batch 65,536, lr 1e-2); m = 1.25, tau = 1024.

One step = the whole job on one resident input: sample + labels, training, prediction, partition,
rounds, polish, merge/repair. Each timed step sorts its own copy of the input (1 GiB, larger than
L2), so no L2 flush is needed. `value` is keys sorted per second over the whole job; the sort alone,
the plain binary32 form, the roofline of the dominant kernel, an end-to-end figure through the
host-array C entry point and the CPU oracle on a bounded sample are reported beside it, and so are
the other workloads (1M uniform keys; 64M uint64 keys with payload; a batch of 4,096 arrays against
one sort call per array; the serving loop), the ablation of the learned map and library CPU sorts.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
  python bench.py --experiment shift|quickdraw|eps   (the paper's Exp-3, Exp-2 stand-in, Exp-4)
  python bench.py --serve-full                        (the serving loop alone)
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_KEYS = 268_435_456
ARCH = dict(layers=2, h1=64, h2=64)
TRAIN = dict(translate="ordbits", sample_n=N_KEYS // 100, steps=100, batch=65536, lr=1e-2, seed=0)
SORT = dict(m=1.25, eps=3, tau=1024)
WORKLOAD = ("268,435,456 float32 keys lognormal(0,2) with 5% exact duplicates, keys only; "
            "MLP 1-64-64-1 trained on the device (1% sample, 100 Adam steps, batch 65536, lr 1e-2); "
            "m=1.25, tau=1024; bucket width, polish blocks per SM and eps from the autotuned table")

# DRAM bytes per key of one launch (dram__bytes_read.sum + dram__bytes_write.sum over the keys of
# the launch) from single-kernel ncu captures at 2^26 keys of the same distribution and model
# recipe; traffic grows in proportion to the keys. A kernel changed since its capture has no entry.
TRAFFIC_PER_KEY = {
    ("predict", "bf16x2"): 7.363,   # k_predict_bf16_mg<64, split>
    ("partition", None): 19.78,     # per pass: k_tile_hist 4.22 + k_scatter 15.56
    ("rounds", None): 6.79,         # k_rounds
    ("polish", None): 12.58,        # k_polish
}
TRAFFIC_SOURCE = "ncu capture of the kernel at 2^26 keys, scaled to the launch's keys"
# binary32 operations per key on the CUDA cores in the tensor-core predict (layer 1: H FMA; split
# form: H residual subtractions; output layer: H additions and H FMA; FMA = 2)
CUDA_CORE_FLOP_PER_KEY = {"bf16": 2 * 64 + 64 + 2 * 64, "bf16x2": 2 * 64 + 64 + 64 + 2 * 64}


def mlp_flop_per_key(layers, h1, h2):
    """The method's own work per key evaluation: 2 (fan-in x fan-out) summed over the layers."""
    return 2 * (h1 + h1 * h2 + h2) if layers == 2 else 2 * (h1 + h1)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm_gbs": p["hbm_gbs"], "bf16_tflops": p["bf16_tflops"],
                "bf16_tflops_sustained": p.get("bf16_tflops_sustained", p["bf16_tflops"]),
                "sm_max_mhz": p.get("sm_max_mhz", 2070.0), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0, "source": "fallback"}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.p = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        # the sampler takes a moment to start: let its first row arrive (at most 3 s) so that the
        # timed region that follows is sampled
        t0 = time.perf_counter()
        while self.p is not None and self.p.poll() is None and time.perf_counter() - t0 < 3.0:
            try:
                if os.path.getsize(self.f.name) > 0:
                    break
            except OSError:
                break
            time.sleep(0.01)
        self.skip = 0
        try:
            self.skip = len([r for r in open(self.f.name).read().splitlines() if r.strip()])
        except OSError:
            pass
        return self

    def __exit__(self, *a):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        try:
            rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        except Exception:
            rows = []
        # rows logged before the timed region opened are not counted, unless there is nothing else
        if len(rows) > getattr(self, "skip", 0):
            rows = rows[getattr(self, "skip", 0):]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4)
                          if len(r) > 5 + i and r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def dist_setup():
    import torch
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, ws: int) -> float:
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- CPU oracle leg
def oracle_job(n: int, seed: int = 2):
    """The oracle as it stands: binary64 training on a 1% sample + sequential NN-sort."""
    import workloads as W
    from oracle import oracle as orc
    keys = W.lognormal_dup_f32(n, seed=seed, sigma=2.0)
    t0 = time.perf_counter()
    model, _, _ = orc.train(keys, ARCH["layers"], ARCH["h1"], ARCH["h2"], orc.ORDBITS,
                            sample_n=max(1, n // 100), steps=100, batch=0, lr=1e-2, seed=0)
    out, _, _, _ = orc.nnsort_model(keys, model, SORT["m"], SORT["eps"], SORT["tau"])
    dt = time.perf_counter() - t0
    return n / dt / 1e6, dt


def reference_arm(args, ws, rank):
    if rank != 0:
        return
    n = 100_000
    for _ in range(args.warmup):
        oracle_job(n)
    t = 0.0
    for _ in range(args.steps):
        _, dt = oracle_job(n)
        t += dt
    v = n * args.steps / t / 1e6
    line = {"impl": "reference", "metric": "Mkeys/s", "value": v, "unit": "Mkeys/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "reference_sample_keys": n},
            "cpu_baseline": {"value": v, "unit": "Mkeys/s", "cores": 1, "kind": "oracle",
                             "sample": f"{n} keys of the same distribution per step, same model "
                                       "and training recipe (1% sample, 100 full-batch steps)"},
            "e2e": {"value": v, "unit": "Mkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- serving leg
SERVE_TRAIN = dict(layers=2, h1=32, h2=32, sample_n=20_000, steps=100, batch=4096, lr=1e-2)


def _serve_once(nns, reqs, scale, workers, max_batch):
    """One pass of the request stream through a server: arrivals at reqs' times x `scale` (0 = all
    at once), each request's array copied fresh. Returns (latencies s, wall s)."""
    arrays = [r["keys"].copy() for r in reqs]
    lats = []
    with nns.Server(hbm_budget=120 << 30, train=SERVE_TRAIN, workers=workers,
                    max_batch=max_batch) as srv:
        t0 = time.perf_counter()
        tickets = []
        for i, r in enumerate(reqs):
            dt = r["arrival_s"] * scale - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(arrays[i], seed=i))
        for t in tickets:
            _, lat = srv.wait(t)
            lats.append(lat)
        wall = time.perf_counter() - t0
    for i in range(0, len(reqs), max(1, len(reqs) // 8)):
        assert np.all(arrays[i][1:] >= arrays[i][:-1])
    return lats, wall


def serving_leg(nns, W, count=1000, lo=10_000, hi=16_000_000, repeats=3, seed=5):
    """float64 requests (log-uniform sizes in [lo, hi]; uniform / lognormal(0,2) / clustered),
    per-request device-trained 1-32-32-1, 120 GiB admission budget. First a saturation run (every
    request submitted at once, continuous batching) gives the saturated request rate; then Poisson
    arrivals at 0.7 x that rate through continuous batching (2 worker streams, up to 16 requests
    per batch), `repeats` times, and once through FIFO (1 worker, 1 request per batch). Latency:
    submit -> sorted result back in host memory."""
    reqs = W.serving_requests(count=count, seed=seed, lo=lo, hi=hi, rate_per_s=1.0)
    keys = int(sum(r["keys"].shape[0] for r in reqs))
    _, wall = _serve_once(nns, reqs, 0.0, 2, 16)
    sat_rate = count / wall
    rate = 0.7 * sat_rate
    scale = 1.0 / rate  # arrivals were drawn at 1 request/s
    out = {"requests": count, "sizes": [lo, hi], "keys": keys,
           "saturated": {"requests_per_s": sat_rate, "mkeys_s": keys / wall / 1e6},
           "offered_rate_per_s": rate}
    runs = []
    for _ in range(repeats):
        lats, wall = _serve_once(nns, reqs, scale, 2, 16)
        runs.append({"p50_ms": 1e3 * float(np.percentile(lats, 50)),
                     "p99_ms": 1e3 * float(np.percentile(lats, 99)), "mkeys_s": keys / wall / 1e6})
    out["continuous_batching"] = {
        "runs": runs, "p50_ms_median": statistics.median(r["p50_ms"] for r in runs),
        "p99_ms_median": statistics.median(r["p99_ms"] for r in runs),
        "mkeys_s_median": statistics.median(r["mkeys_s"] for r in runs)}
    lats, wall = _serve_once(nns, reqs, scale, 1, 1)
    out["fifo"] = {"p50_ms": 1e3 * float(np.percentile(lats, 50)),
                   "p99_ms": 1e3 * float(np.percentile(lats, 99)), "mkeys_s": keys / wall / 1e6}
    return out


def serving_full(nns, W):
    return serving_leg(nns, W, count=1000)


# --------------------------------------------------------------------------- experiments
# Sec. "Experimental Study" beside the headline job: each prints one JSON line per setting.
PAPER_RECIPE = dict(layers=2, h1=2, h2=6, loss="huber", huber_delta=0.01, batch=128, lr=1e-3,
                    steps=2000)  # three hidden layers of 2, 6 and 1 neurons, Eq. (loss), batch 128


def _sorted_ms(nns, torch, src, model, precision, reps=3, **sopts):
    """Median sort time (the library's stage events), the last run's statistics, and whether the
    output equals torch.sort of the input."""
    work = torch.empty_like(src)
    ms, st = [], None
    for _ in range(reps):
        work.copy_(src)
        torch.cuda.synchronize()
        st = nns.sort(work, None, model, precision=precision, timing=True, **sopts)
        ms.append(st["ms_stage"][7])
    return statistics.median(ms), st, work


def _library_sort_ms(torch, src, reps=3):
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(reps):
        torch.cuda.synchronize()
        a.record(s)
        out = torch.sort(src).values
        b.record(s)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    return statistics.median(ms), out


def _host_sort_rate(keys, cap=4_000_000):
    sample = np.array(keys[:cap])
    t0 = time.perf_counter()
    np.sort(sample, kind="quicksort")
    return sample.shape[0] / (time.perf_counter() - t0) / 1e6


def _form(n, ms, st):
    return {"sort_ms": ms, "mkeys_s": n / (ms / 1e3) / 1e6, "rounds": st["t"],
            "sigma": st["sigma"], "trad_rate": st["trad_rate"], "repaired": st["repaired"]}


def experiment_shift(nns, W, torch):
    """Exp-3: f (1-32-1, 1% sample, 100 Adam steps, lr 1e-2) trained once on 26,214,400 uniform
    float32 keys (100 MB), then used unchanged to sort inputs of the same size with 0..60% of the
    keys replaced by normal(0.5, 0.1) noise; torch.sort (the library's radix sort) and numpy's sort
    on one host core beside it."""
    from paper_1907_08817_gb300 import autotune as AT
    n = 26_214_400
    tk = torch.from_numpy(W.uniform_f32(n, 0)).cuda()
    model, _ = nns.train(tk, layers=1, h1=32, h2=0, sample_n=n // 100, steps=100, batch=0, lr=1e-2,
                         seed=0)
    del tk
    for noise in (0.0, 0.15, 0.30, 0.45, 0.60):
        host = W.shift_mix_f32(n, noise, seed=6)
        src = torch.from_numpy(host).cuda()
        lib_ms, ref = _library_sort_ms(torch, src)
        forms = {}
        for prec in ("fp32", "pwl"):
            o = AT.tuned_options(0, n, 1, 32, 0, prec)
            ms, st, out = _sorted_ms(nns, torch, src, model, prec, **o)
            assert torch.equal(out, ref), "sorted output differs from torch.sort"
            forms[prec] = _form(n, ms, st)
        print(json.dumps({"experiment": "distribution shift (Exp-3)", "n": n, "noise": noise,
                          "model": "1-32-1 trained on uniform keys", "nnsort": forms,
                          "torch_sort_ms": lib_ms, "torch_sort_mkeys_s": n / (lib_ms / 1e3) / 1e6,
                          "host_numpy_sort_mkeys_s": _host_sort_rate(host)}), flush=True)
        del src, ref


def experiment_quickdraw(nns, W, torch):
    """Exp-2's size: 50,426,265 uniform uint64 keys stand in for the QuickDraw key-ids (not
    available here); f 1-32-1 trained on a 1% sample of them (100 Adam steps, lr 1e-2)."""
    from paper_1907_08817_gb300 import autotune as AT
    n = W.QUICKDRAW_RECORDS
    host = W.uniform_u64(n, seed=7)
    src = torch.from_numpy(host.view(np.int64)).cuda()
    s = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(s)
    model, _ = nns.train(src, key_type="u64", layers=1, h1=32, h2=0, sample_n=n // 100, steps=100,
                         batch=0, lr=1e-2, seed=0)
    b.record(s)
    torch.cuda.synchronize()
    train_ms = a.elapsed_time(b)
    flip = torch.tensor(-(1 << 63), dtype=torch.int64, device=src.device)
    lib_ms, ref = _library_sort_ms(torch, src ^ flip)  # unsigned order as signed
    forms = {}
    for prec in ("fp32", "pwl"):
        o = AT.tuned_options(3, n, 1, 32, 0, prec)
        work = torch.empty_like(src)
        ms = []
        for _ in range(3):
            work.copy_(src)
            torch.cuda.synchronize()
            st = nns.sort(work, None, model, precision=prec, timing=True, key_type="u64", **o)
            ms.append(st["ms_stage"][7])
        assert torch.equal(work ^ flip, ref), "sorted output differs from torch.sort"
        f = _form(n, statistics.median(ms), st)
        f["job_mkeys_s"] = n / ((train_ms + f["sort_ms"]) / 1e3) / 1e6
        forms[prec] = f
    print(json.dumps({"experiment": "QuickDraw-sized stand-in (Exp-2)", "n": n,
                      "keys": "uint64 uniform over [0, 2^64)", "train_ms": train_ms,
                      "nnsort": forms, "torch_sort_ms": lib_ms,
                      "torch_sort_mkeys_s": n / (lib_ms / 1e3) / 1e6,
                      "host_numpy_sort_mkeys_s": _host_sort_rate(host)}), flush=True)


def experiment_eps(nns, W, torch, n, precision):
    """Exp-4 with the cost model: the headline input sorted with eps = 1..5 under two models (the
    paper's recipe and the headline one); per eps the sort time, the measured counts (elements
    entering each iteration, the final conflict array, out-of-order elements) and the cost model's
    T(n, e, sigma, t, theta) and counts from the measured sigma_i, e_i."""
    from paper_1907_08817_gb300 import autotune as AT
    from paper_1907_08817_gb300 import costmodel as CM
    src = torch.from_numpy(W.lognormal_dup_f32(n, seed=2, sigma=2.0)).cuda()
    ref = torch.sort(src).values
    for label, arch, rec, prec in (("paper recipe 1-2-6-1", (2, 2, 6), PAPER_RECIPE, "fp32"),
                                   ("headline 1-64-64-1", (2, 64, 64),
                                    dict(**ARCH, **{k: v for k, v in TRAIN.items()
                                                    if k not in ("translate", "seed")}), precision)):
        rec = {**rec, "sample_n": max(1, n // 100)}
        model, hist = nns.train(src, seed=0, **rec)
        o = AT.tuned_options(0, n, *arch, prec)
        theta = 2 * (arch[1] + arch[1] * arch[2] + arch[2]) if arch[0] == 2 else 4 * arch[1]
        for eps in (1, 2, 3, 4, 5):
            ms, st, out = _sorted_ms(nns, torch, src, model, prec, eps=eps,
                                     bucket_log2=o["bucket_log2"], polish_blocks=o["polish_blocks"])
            assert torch.equal(out, ref), "sorted output differs from torch.sort"
            t = st["t"]
            w = st["w_size"]
            sig = [w[i + 1] / w[i] for i in range(t)]
            e = list(st["e"][:t])
            pc = CM.predicted_counts(n, sig, e)
            print(json.dumps({
                "experiment": "iterations and cost model (Exp-4)", "model": label,
                "final_train_loss": float(hist[-1]), "precision": prec, "n": n, "eps": eps,
                "sort_ms": ms, "mkeys_s": n / (ms / 1e3) / 1e6, "t": t,
                "measured": {"entering": w[:t], "leftover": w[t],
                             "out_of_order": st["out_of_order"][:t], "sigma": sig, "e": e},
                "cost_model": {"theta": theta, "entering": pc["entering"],
                               "leftover": pc["leftover"], "out_of_order": pc["out_of_order"],
                               "T_printed": CM.operations(n, sig, e, theta, "printed"),
                               "T_entering": CM.operations(n, sig, e, theta, "entering"),
                               "n_log2_n": CM.quicksort_operations(n)}}), flush=True)
        del model


# --------------------------------------------------------------------------- shared pieces
STAGES = ["predict", "partition", "bucket_bounds", "rounds", "finalize", "polish", "seam"]


def _ev(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def tuned(dtype, n, arch, precision, m=1.25, tau=1024):
    """m and tau as the paper sets them; bucket width, polish blocks per SM and the round limit eps
    from the autotuner's table for this workload class."""
    from paper_1907_08817_gb300 import autotune as AT
    return dict(m=m, tau=tau, **AT.tuned_options(dtype, n, *arch, precision))


def fastest_tensor_form(dtype, n, arch):
    """The tensor-core form the autotuner measured faster on this workload class."""
    from paper_1907_08817_gb300 import autotune as AT
    cands = [(e["sort_ms"], p) for p in ("bf16x2", "bf16")
             if (e := AT.tuned_entry(dtype, n, *arch, p)) is not None]
    return min(cands)[1] if cands else "bf16x2"


def roofline_of(stage, ms, n, kb, pb, precision, arch, npass, pk):
    """Roofline entry of one stage of the sort: its algorithmic work for one launch over its mean
    event time, against the measured peak of the unit that bounds it."""
    traffic = None
    tpk = TRAFFIC_PER_KEY.get((stage, precision), TRAFFIC_PER_KEY.get((stage, None)))
    if tpk is not None and pb == 0 and kb == 4:
        traffic = tpk * n * (npass if stage == "partition" else 1)
    fp32_peak = 152 * 128 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12
    if stage == "predict" and precision in ("bf16", "bf16x2") and arch[0] == 2:
        fpk = mlp_flop_per_key(*arch)
        ach = n * fpk / (ms / 1e3) / 1e12
        peak = pk["bf16_tflops_sustained"]
        r = {"kernel": f"predict (k_predict_bf16_mg, {precision})", "bound": "tensor",
             "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
             "peak_kind": f"bf16 sustained, {pk['source']} (the kernel runs inside a long step)",
             "frac_of_burst": ach / pk["bf16_tflops"],
             "work": f"{fpk} FLOP per key (2 x fan-in x fan-out over the layers) x {n} keys",
             "cuda_cores": {"flop_per_key": CUDA_CORE_FLOP_PER_KEY[precision],
                            "achieved": n * CUDA_CORE_FLOP_PER_KEY[precision] / (ms / 1e3) / 1e12,
                            "peak": fp32_peak, "unit": "TFLOP/s",
                            "peak_source": "152 SMs x 128 FP32 lanes x 2 FLOP x max SM clock"}}
        r["cuda_cores"]["frac"] = r["cuda_cores"]["achieved"] / fp32_peak
    elif stage == "predict" and precision == "fp32":
        fpk = mlp_flop_per_key(*arch)
        ach = n * fpk / (ms / 1e3) / 1e12
        r = {"kernel": "predict (k_predict, binary32 FFMA)", "bound": "alu", "achieved": ach,
             "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
             "peak_kind": "152 SMs x 128 FP32 lanes x 2 FLOP x max SM clock",
             "work": f"{fpk} FLOP per key x {n} keys"}
    else:
        per = {"predict": kb + 4 + pb, "partition": npass * 2 * (kb + 4 + pb),
               "bucket_bounds": 0, "rounds": kb + 4 + 1, "finalize": 0,
               "polish": 2 * kb + 5 + 2 * pb, "seam": 0}[stage]
        ach = n * per / (ms / 1e3) / 1e9
        r = {"kernel": stage, "bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"],
             "unit": "GB/s", "frac": ach / pk["hbm_gbs"], "peak_kind": f"copy bandwidth, {pk['source']}",
             "work": f"{per} algorithmic bytes per key x {n} keys"}
    r["ms"] = ms
    r["traffic"] = traffic
    r["traffic_source"] = TRAFFIC_SOURCE if traffic is not None else None
    return r


def path_of(st, n, kb, pb, sort_ms, pk):
    """The whole sort against the path's algorithmic bytes: four passes over every element (read,
    place, read back, write) and three more per re-mapped conflict."""
    w = st["w_size"]
    b_alg = 4 * n * (kb + pb) + 3 * sum(w[1:-1]) * (kb + pb) if len(w) > 2 else 4 * n * (kb + pb)
    return {"b_alg_bytes": b_alg, "sort_ms": sort_ms,
            "frac": b_alg / (sort_ms / 1e3) / 1e9 / pk["hbm_gbs"],
            "frac_of_8tbs": b_alg / (sort_ms / 1e3) / 1e9 / 8000.0}


def _timed_sorts(nns, torch, src, model, precision, opts, reps=2, payload=None, key_type=None):
    """(median sort ms from the library's stage events, the last run's statistics, the output)."""
    work = torch.empty_like(src)
    wp = None if payload is None else torch.empty_like(payload)
    ms, st = [], None
    for _ in range(reps):
        work.copy_(src)
        if wp is not None:
            wp.copy_(payload)
        torch.cuda.synchronize()
        st = nns.sort(work, wp, model, precision=precision, timing=True, key_type=key_type, **opts)
        ms.append(st["ms_stage"][7])
    return statistics.median(ms), st, work, wp


def _form_entry(n, ms, st, train_ms=None):
    e = {"sort_ms": ms, "sort_mkeys_s": n / (ms / 1e3) / 1e6, "rounds": st["t"],
         "sigma": st["sigma"], "trad_rate": st["trad_rate"], "repaired": st["repaired"],
         "oversized_buckets": st["oversized_buckets"],
         "stage_ms": dict(zip(STAGES, st["ms_stage"][:7]))}
    if train_ms is not None:
        e["job_ms"] = train_ms + ms
        e["job_mkeys_s"] = n / ((train_ms + ms) / 1e3) / 1e6
    return e


def _e2e_host(nns, L, torch, host, payload, dtype, arch, train, precision, so, reps=3):
    """End to end through nnsort_train_sort_host from pinned host arrays: copies in, device
    training, sort, copies out, all inside the timed call."""
    import ctypes as C
    hk = torch.from_numpy(host.view({4: np.int32, 8: np.int64}[host.dtype.itemsize]).copy()).pin_memory()
    hp = None if payload is None else torch.from_numpy(payload.copy()).pin_memory()
    to = nns._topts(**arch, **train)
    sop = nns._sopts(so["m"], so["eps"], so["tau"], precision, so["bucket_log2"], None, None, False,
                     False, so["polish_blocks"])
    s = torch.cuda.current_stream()
    tt = []
    for k in range(reps + 1):
        hk.numpy()[:] = host.view(hk.numpy().dtype)
        if hp is not None:
            hp.numpy()[:] = payload
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc = L.lib().nnsort_train_sort_host(C.c_void_p(hk.data_ptr()),
                                            None if hp is None else C.c_void_p(hp.data_ptr()),
                                            host.shape[0], dtype, C.byref(to), C.byref(sop), None,
                                            None, C.c_void_p(s.cuda_stream))
        t1 = time.perf_counter()
        L.check("nnsort_train_sort_host", rc)
        if k:
            tt.append(t1 - t0)
    n = host.shape[0]
    pb = 0 if payload is None else 4
    return {"value": n / statistics.median(tt) / 1e6, "unit": "Mkeys/s",
            "h2d_bytes_per_step": n * (host.dtype.itemsize + pb),
            "d2h_bytes_per_step": n * (host.dtype.itemsize + pb)}


# --------------------------------------------------------------------------- other workloads
C1_TRAIN = dict(translate="ordbits", sample_n=10_000, steps=100, batch=0, lr=1e-2, seed=0)


def leg_c1(nns, W, torch, L, pk, steps=20, warmup=3):
    """1,000,000 float32 keys U[0,1) (seed 0), keys only; 1-32-1 in binary32 trained on a 1% sample
    (100 full-batch Adam steps, lr 1e-2). One step = training + sort, each on its own copy."""
    n, arch = 1_000_000, (1, 32, 0)
    A = dict(layers=1, h1=32, h2=0)
    host = W.uniform_f32(n, 0)
    src = torch.from_numpy(host).cuda()
    so = tuned(0, n, arch, "fp32")
    bufs = [src.clone() for _ in range(warmup + steps)]
    l0 = L.lib().nnsort_launch_count()

    def job(b):
        model, _ = nns.train(b, **A, **C1_TRAIN)
        nns.sort(b, None, model, precision="fp32", stats=False, **so)
    for k in range(warmup):
        job(bufs[k])
    torch.cuda.synchronize()
    l0 = L.lib().nnsort_launch_count()
    a, b = _ev(torch)
    a.record()
    for k in range(steps):
        job(bufs[warmup + k])
    b.record()
    torch.cuda.synchronize()
    launches = (L.lib().nnsort_launch_count() - l0) / steps
    ms = a.elapsed_time(b) / steps
    ref = torch.sort(src).values
    assert all(torch.equal(bufs[warmup + k], ref) for k in range(steps)), "c1 output differs"
    model, _ = nns.train(src, **A, **C1_TRAIN)
    ta, tb = _ev(torch)
    ta.record()
    nns.train(src, **A, **C1_TRAIN)
    tb.record()
    torch.cuda.synchronize()
    train_ms = ta.elapsed_time(tb)
    sms, st, out, _ = _timed_sorts(nns, torch, src, model, "fp32", so, reps=5)
    assert torch.equal(out, ref)
    pms, pst, out, _ = _timed_sorts(nns, torch, src, model, "pwl", tuned(0, n, arch, "pwl"), reps=5)
    assert torch.equal(out, ref)
    return {"workload": "1,000,000 float32 keys U[0,1) seed 0, keys only; MLP 1-32-1 binary32 "
                        "trained on the device (1% sample, 100 full-batch Adam steps, lr 1e-2)",
            "value": n / ms / 1e3, "unit": "Mkeys/s", "ms_per_step": ms, "steps": steps,
            "warmup": warmup, "precision": "fp32", "sort_opts": so, "train_ms": train_ms,
            "launches_per_step": launches,
            "bound": "launch and latency: the 4 MB input and every buffer fit in L2, so the HBM "
                     "roofline fraction is not a meaningful bound here",
            "sort": _form_entry(n, sms, st), "compiled_form": _form_entry(n, pms, pst),
            "path": path_of(st, n, 4, 0, sms, pk),
            "e2e": _e2e_host(nns, L, torch, host, None, 0, A, C1_TRAIN, "fp32", so),
            "parity": "every timed output equals torch.sort of the input (bit for bit)"}


C3_ARCH = dict(layers=2, h1=32, h2=32)
C3_TRAIN = dict(translate="ordbits", sample_n=1_048_576, steps=200, batch=65536, lr=1e-2, seed=0)


def leg_c3(nns, W, torch, L, pk, steps=5, warmup=3):
    """67,108,864 uint64 keys from a Zipf(1.1)-weighted mixture of 8 Gaussians over [0, 2^63), each
    with an int32 payload (its index), stable key-value sort; 1-32-32-1 trained on the device on a
    1,048,576-key sample (200 Adam steps, mini-batch 65,536, lr 1e-2). One step = training + sort."""
    n, arch = 1 << 26, (2, 32, 32)
    keys, payload = W.gauss_mix_u64(n, 3)
    sk = torch.from_numpy(keys.view(np.int64)).cuda()
    sp = torch.from_numpy(payload).cuda()
    prec = fastest_tensor_form(3, n, arch)
    so = tuned(3, n, arch, prec)
    bk = [sk.clone() for _ in range(warmup + steps)]
    bp = [sp.clone() for _ in range(warmup + steps)]

    def job(k, p):
        model, hist = nns.train(k, key_type="u64", **C3_ARCH, **C3_TRAIN)
        nns.sort(k, p, model, precision=prec, stats=False, key_type="u64", **so)
        return hist
    for k in range(warmup):
        hist = job(bk[k], bp[k])
    torch.cuda.synchronize()
    l0 = L.lib().nnsort_launch_count()
    a, b = _ev(torch)
    a.record()
    for k in range(steps):
        job(bk[warmup + k], bp[warmup + k])
    b.record()
    torch.cuda.synchronize()
    launches = (L.lib().nnsort_launch_count() - l0) / steps
    ms = a.elapsed_time(b) / steps
    flip = torch.tensor(-(1 << 63), dtype=torch.int64, device="cuda")
    rv, ri = torch.sort(sk ^ flip, stable=True)
    rv ^= flip
    ri = ri.to(torch.int32)
    for k in range(steps):
        assert torch.equal(bk[warmup + k], rv) and torch.equal(bp[warmup + k], ri), "c3 differs"
    del bk, bp
    ta, tb = _ev(torch)
    ta.record()
    model, hist = nns.train(sk, key_type="u64", **C3_ARCH, **C3_TRAIN)
    tb.record()
    torch.cuda.synchronize()
    train_ms = ta.elapsed_time(tb)
    forms = {}
    for p_ in dict.fromkeys((prec, "fp32", "pwl")):
        o = tuned(3, n, arch, p_)
        fms, fst, out, outp = _timed_sorts(nns, torch, sk, model, p_, o, reps=3, payload=sp,
                                           key_type="u64")
        assert torch.equal(out, rv) and torch.equal(outp, ri)
        forms[p_] = dict(_form_entry(n, fms, fst, train_ms), sort_opts=o)
        if p_ == prec:
            st_c, ms_c = fst, fms
    live = {k_: v for k_, v in zip(STAGES, st_c["ms_stage"][:7])}
    dom = max(STAGES, key=lambda k_: live[k_])
    return {"workload": "67,108,864 uint64 keys, mixture of 8 Gaussians (Zipf 1.1 weights, means over "
                        "[0, 2^63)), int32 payload = index, stable key-value; MLP 1-32-32-1 trained on "
                        "the device (1,048,576-key sample, 200 Adam steps, batch 65536, lr 1e-2)",
            "value": n / ms / 1e3, "unit": "Mkeys/s", "ms_per_step": ms, "steps": steps,
            "warmup": warmup, "precision": prec, "sort_opts": so, "train_ms": train_ms,
            "final_train_loss": float(hist[-1]), "launches_per_step": launches,
            "forms": forms,
            "roofline": roofline_of(dom, live[dom], n, 8, 4, prec, arch,
                                    st_c["partition_passes"], pk),
            "path": path_of(st_c, n, 8, 4, ms_c, pk),
            "e2e": _e2e_host(nns, L, torch, keys, payload, 3, C3_ARCH, C3_TRAIN, prec, so, reps=2),
            "parity": "every timed output equals torch.sort (stable) of the keys; payloads equal "
                      "its stable permutation"}, model, sk


C4_TRAIN = dict(translate="ordbits", steps=100, batch=0, lr=1e-2)


def leg_c4(nns, W, torch, L, pk, reps=3):
    """4,096 float32 arrays, sizes floor(1000 * 1000^U), each from uniform / normal / lognormal /
    exponential, each with its own 1-16-1 (1% sample, 100 full-batch Adam steps, lr 1e-2): the
    batched sort (one pipeline pass over every array) against one nnsort_sort call per array, on
    the same inputs and models."""
    arrs = [a for _, a in W.batch_arrays(4096, seed=4)]
    sizes = [a.shape[0] for a in arrs]
    total = int(sum(sizes))
    src = torch.from_numpy(np.concatenate(arrs)).cuda()
    del arrs
    offs = np.concatenate([[0], np.cumsum(sizes)])
    views = lambda t: [t[offs[j]:offs[j + 1]] for j in range(len(sizes))]  # noqa: E731
    sv = views(src)
    sample_ns = [max(1, v.numel() // 100) for v in sv]
    tms = {}
    for label, batched in (("batch", True), ("loop", False), ("batch", True)):
        ta, tb = _ev(torch)
        ta.record()
        if batched:
            models, _ = nns.train_batch(sv, sample_ns=sample_ns, layers=1, h1=16, h2=0, seed=0,
                                        **C4_TRAIN)
        else:
            loop_models = [nns.train(v, layers=1, h1=16, h2=0, sample_n=sample_ns[j], seed=j,
                                     **C4_TRAIN)[0] for j, v in enumerate(sv)]
        tb.record()
        torch.cuda.synchronize()
        tms[label] = ta.elapsed_time(tb)  # the second batched run is the one kept (warm)
    # the batched models follow the same recipe and seeds as the loop's (their sums run in another
    # order, so the weights agree to training noise): the largest weight difference, relative
    wdiff = 0.0
    for j in range(0, len(sv), 512):
        d0, p0 = models[j].describe()
        d1, p1 = loop_models[j].describe()
        assert d0 == d1, "batched training used another sample"
        wdiff = max(wdiff, float(np.max(np.abs(p0 - p1)) / max(np.abs(p1).max(), 1e-30)))
    del loop_models
    train_ms = tms["batch"]
    so = tuned(0, total // len(sizes), (1, 16, 0), "fp32")
    work = torch.empty_like(src)
    wv = views(work)
    refs = [torch.sort(v).values for v in sv]

    def run(batch):
        work.copy_(src)
        torch.cuda.synchronize()
        a, b = _ev(torch)
        a.record()
        if batch:
            nns.sort_batch(wv, models, precision="fp32", stats=False, **so)
        else:
            for v, f in zip(wv, models):
                nns.sort(v, None, f, precision="fp32", stats=False, **so)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)
    out = {}
    for label, batch, k in (("batch", True, reps), ("loop", False, max(1, reps - 1))):
        run(batch)  # warm-up
        l0 = L.lib().nnsort_launch_count()
        ms = [run(batch) for _ in range(k)]
        launches = (L.lib().nnsort_launch_count() - l0) / k
        assert all(torch.equal(o, r) for o, r in zip(wv, refs)), f"c4 {label} output differs"
        out[label] = {"ms": statistics.median(ms), "mkeys_s": total / (statistics.median(ms) / 1e3) / 1e6,
                      "launches": launches}
    st = nns.sort_batch(wv, models, precision="fp32", **so)
    sig = [s_["sigma"][0] for s_ in st if s_["t"]]
    job_ms = train_ms + out["batch"]["ms"]
    return {"workload": "4,096 float32 arrays, sizes log-uniform in [1K, 1M] (seed 4), each uniform / "
                        "normal / lognormal / exponential, per-array MLP 1-16-1 (1% sample, 100 Adam "
                        "steps, lr 1e-2)",
            "arrays": len(sizes), "keys": total,
            "value": total / (job_ms / 1e3) / 1e6, "unit": "Mkeys/s",
            "job": "batched training of every model + one batched sort",
            "job_ms": job_ms, "sort": out["batch"], "sort_loop_one_call_per_array": out["loop"],
            "sort_batch_speedup": out["loop"]["ms"] / out["batch"]["ms"], "sort_opts": so,
            "train_ms": {"batched (nnsort_train_batch)": tms["batch"],
                         "one nnsort_train call per array": tms["loop"]},
            "sigma_1_median": float(np.median(sig)) if sig else None,
            "train_weight_diff_batched_vs_loop": wdiff,
            "parity": "every array of both sorts equals torch.sort of that array (bit for bit); "
                      "the batched models use the same samples and normalisers as nnsort_train's"}


def ablation(nns, torch, src, model, n, kb, arch, key_type, dtype, chosen, pk):
    """What the learned map gains (Sec. "Experimental Study", Exp-1 and Exp-5): the same pipeline
    with the linear min-max map F(x) = x (no learning; in the key's value and in its order image),
    the untrained network (initial weights), the learned network in each form, and a radix sort of
    every key (no model) -- sigma_1, traditional sorting rate, seam repairs and sort time each."""
    d, _ = model.describe()
    if key_type == "u64":
        flip = torch.tensor(-(1 << 63), dtype=torch.int64, device="cuda")
        fl = src ^ flip
        vlo = float(int((fl.min() ^ flip).item()) & ((1 << 64) - 1))
        vhi = float(int((fl.max() ^ flip).item()) & ((1 << 64) - 1))
        del fl
    else:
        vlo, vhi = float(src.min().item()), float(src.max().item())
    lin_value = nns.Model.create(dtype, 1, 1, 0, [1.0, 0.0, 1.0, 0.0], "value", 0, vlo,
                                 1.0 / (vhi - vlo) if vhi > vlo else 1.0)
    lin_order = nns.Model.create(dtype, 1, 1, 0, [1.0, 0.0, 1.0, 0.0], "ordbits", d["lo_bits"],
                                 d["lo_val"], d["scale"])
    untrained, _ = nns.train(src, key_type=key_type, layers=arch[0], h1=arch[1], h2=arch[2],
                             sample_n=max(1, n // 100), steps=0, seed=0)
    if key_type == "u64":
        ref = torch.sort(src ^ flip).values ^ flip
    else:
        ref = torch.sort(src).values
    out = {}
    for label, f, prec, a_ in (("linear map, key value", lin_value, "fp32", (1, 1, 0)),
                               ("linear map, order image", lin_order, "fp32", (1, 1, 0)),
                               ("untrained network", untrained, "fp32", arch),
                               ("learned network, binary32", model, "fp32", arch),
                               (f"learned network, {chosen}", model, chosen, arch),
                               ("learned network, compiled", model, "pwl", arch)):
        o = tuned(dtype, n, arch, prec)
        ms, st, w, _ = _timed_sorts(nns, torch, src, f, prec, o, reps=2, key_type=key_type)
        assert torch.equal(w, ref), label
        out[label] = {"sort_ms": ms, "sort_mkeys_s": n / (ms / 1e3) / 1e6,
                      "sigma_1": st["sigma"][0] if st["t"] else None, "trad_rate": st["trad_rate"],
                      "repaired": st["repaired"], "oversized_buckets": st["oversized_buckets"]}
    work = torch.empty_like(src)
    ms = []
    for _ in range(2):
        work.copy_(src)
        torch.cuda.synchronize()
        a, b = _ev(torch)
        a.record()
        nns.radix_sort(work, key_type=key_type)
        b.record()
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
    assert torch.equal(work, ref)
    out["no model: radix sort of every key (nnsort_radix_sort)"] = {
        "sort_ms": statistics.median(ms), "sort_mkeys_s": n / (statistics.median(ms) / 1e3) / 1e6}
    lib_ms, _ = _library_sort_ms(torch, src if key_type != "u64" else src ^ flip)
    out["context: torch.sort (library radix sort)"] = {"sort_ms": lib_ms,
                                                        "sort_mkeys_s": n / (lib_ms / 1e3) / 1e6}
    return out


def cpu_info():
    model = None
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": os.uname().machine}


def cpu_sorts(host, cap=16_777_216):
    """Library CPU sorts of a bounded sample of the headline keys on the host cores."""
    from oracle import oracle as orc
    sample = np.ascontiguousarray(host[:cap])
    res = {"sample": f"first {sample.shape[0]} keys of the headline input", **cpu_info()}
    for label, algo, th in (("std::stable_sort, 1 thread", "stable_sort", 1),
                            ("std::sort, 1 thread", "sort", 1),
                            (f"parallel std::sort + merges, {os.cpu_count()} threads", "parallel",
                             os.cpu_count())):
        _, dt = orc.cpu_sort(sample, algo, th)
        res[label] = {"mkeys_s": sample.shape[0] / dt / 1e6, "seconds": dt, "threads": th}
    return res


# --------------------------------------------------------------------------- GPU arm
def _bf16_rn(a):
    """binary32 -> BF16 (round to nearest even), returned as binary32."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def w2_split_displacement(keys_sample, desc, params, nm):
    """Where the split-BF16 form's displacement comes from, on a host sample of keys (two-layer
    models, float32 keys, order-image translate): F(x) in binary64 with the split form's operands --
    each first-layer activation as a BF16 part (truncated) plus an FP16 rest, W2 as the kernel stages
    it (BF16 for the BF16 part, FP16 for the rest) -- against F(x) with W2 carried as a BF16 part
    plus a BF16 rest, and against exact W2; each against the binary64 model on the same inputs.
    Displacements are |dF| * n * m (positions)."""
    h1, h2 = desc["h1"], desc["h2"]
    p = params.astype(np.float64)
    W1, b1 = p[:h1], p[h1:2 * h1]
    W2 = p[2 * h1:2 * h1 + h1 * h2].reshape(h2, h1)
    b2 = p[2 * h1 + h1 * h2:2 * h1 + h1 * h2 + h2]
    W3 = p[2 * h1 + h1 * h2 + h2:2 * h1 + h1 * h2 + 2 * h2]
    b3 = p[-1]
    w = keys_sample.astype(np.float32).view(np.uint32).astype(np.uint64)
    u = np.where(w & 0x80000000, ~w & 0xFFFFFFFF, w | 0x80000000)  # order image
    lo = int(desc["lo_bits"])
    d = np.where(u >= lo, (u - lo).astype(np.float64), -((lo - u).astype(np.float64)))
    x = (d.astype(np.float32) * np.float32(desc["scale"])).astype(np.float64)
    h = np.maximum(np.outer(x, W1) + b1, 0.0)
    exact = np.maximum(h @ W2.T + b2, 0.0) @ W3 + b3
    h32 = h.astype(np.float32)
    hi = (h32.view(np.uint32) & np.uint32(0xFFFF0000)).view(np.float32).astype(np.float64)
    rest = np.float16(h32.astype(np.float64) - hi).astype(np.float64)
    W2b = _bf16_rn(W2.astype(np.float32)).astype(np.float64)
    W2h = np.float16(W2.astype(np.float32)).astype(np.float64)
    W2r = _bf16_rn((W2.astype(np.float32) - W2b.astype(np.float32))).astype(np.float64)
    out = {"sample_keys": int(keys_sample.size)}
    for name, A, B in (("as the kernel (W2 in BF16 for the BF16 part, FP16 for the rest)", W2b, W2h),
                       ("W2 carried as BF16 part + BF16 rest", W2b + W2r, W2h),
                       ("exact W2 (activations split only)", W2, W2)):
        y = np.maximum(hi @ A.T + rest @ B.T + b2, 0.0) @ W3 + b3
        dd = np.abs(np.clip(y, 0.0, 1.0) - np.clip(exact, 0.0, 1.0)) * nm
        out[name] = {"mean_abs": float(dd.mean()), "max_abs": float(dd.max())}
    return out


def run_job(nns, keys, precision, sopts, stats=True, timing=False):
    model, hist = nns.train(keys, **ARCH, **TRAIN)
    st = nns.sort(keys, None, model, precision=precision, stats=stats, timing=timing, **sopts)
    return model, hist, st


def tuned_sort_opts(precision, n):
    """m and tau as the paper sets them; bucket width, polish blocks per SM and the round limit eps
    from the autotuner's table for this workload class."""
    from paper_1907_08817_gb300 import autotune as AT
    t = AT.tuned_options(0, n, ARCH["layers"], ARCH["h1"], ARCH["h2"], precision)
    return dict(m=SORT["m"], tau=SORT["tau"], **t)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours")
    ap.add_argument("--n", type=int, default=N_KEYS)
    ap.add_argument("--precision", default="auto")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the other workloads")
    ap.add_argument("--no-ablation", action="store_true")
    ap.add_argument("--serve-full", action="store_true",
                    help="only the serving loop (1,000 requests of 10K..16M keys)")
    ap.add_argument("--experiment", choices=["shift", "quickdraw", "eps"], default=None,
                    help="run one of the paper's experiments instead of the benchmark job")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        reference_arm(args, ws, rank)
        return

    import torch
    import paper_1907_08817_gb300 as nns
    import workloads as W
    from paper_1907_08817_gb300 import _lib as L
    torch.cuda.set_device(local)
    n = args.n
    if args.n != N_KEYS:
        TRAIN["sample_n"] = max(1, n // 100)
    if args.experiment is not None:
        if rank == 0:
            if args.experiment == "shift":
                experiment_shift(nns, W, torch)
            elif args.experiment == "quickdraw":
                experiment_quickdraw(nns, W, torch)
            else:
                experiment_eps(nns, W, torch, n,
                               "bf16x2" if args.precision == "auto" else args.precision)
        return
    pk = peaks()
    if args.serve_full:
        if rank == 0:
            print(json.dumps({"serving_full": serving_full(nns, W)}), flush=True)
        return

    host = W.lognormal_dup_f32(n, seed=2, sigma=2.0)
    pristine = torch.from_numpy(host).cuda()
    nbuf = args.steps + args.warmup
    bufs = [pristine.clone() for _ in range(nbuf)]
    torch.cuda.synchronize()

    precision = args.precision
    if precision == "auto":
        precision = fastest_tensor_form(0, n, (ARCH["layers"], ARCH["h1"], ARCH["h2"]))

    sopts = tuned_sort_opts(precision, n)
    s = torch.cuda.current_stream()
    # warm-up
    for k in range(args.warmup):
        run_job(nns, bufs[k], precision, sopts)
    torch.cuda.synchronize()
    # timed region: K whole jobs, each on its own resident input
    launches0 = L.lib().nnsort_launch_count()
    timed_stages = []
    clk = Clocks(local)
    with clk:
        barrier(ws)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for k in range(args.steps):
            # the library records CUDA events around each stage on the call's stream
            timed_stages.append(run_job(nns, bufs[args.warmup + k], precision, sopts,
                                        timing=True)[2]["ms_stage"])
        e1.record(s)
        torch.cuda.synchronize()
        barrier(ws)
    launches = L.lib().nnsort_launch_count() - launches0
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, ws)
    value = ws * n * args.steps / (ms_max / 1e3) / 1e6

    # correctness of the timed outputs (cheap device check)
    ref = torch.sort(pristine).values
    ok = all(torch.equal(bufs[args.warmup + k].view(torch.int32), ref.view(torch.int32))
             for k in range(args.steps))
    assert ok, "sorted output differs from torch.sort"
    del ref

    # breakdown: training vs sort, per-stage timings (separate, untimed-for-value runs)
    job = pristine.clone()
    ta = torch.cuda.Event(enable_timing=True)
    tb = torch.cuda.Event(enable_timing=True)
    ta.record(s)
    model, hist = nns.train(job, **ARCH, **TRAIN)
    tb.record(s)
    torch.cuda.synchronize()
    train_ms = ta.elapsed_time(tb)
    stage_runs = []
    for _ in range(3):
        job.copy_(pristine)
        torch.cuda.synchronize()
        st = nns.sort(job, None, model, precision=precision, timing=True, **sopts)
        stage_runs.append(st["ms_stage"])
    stage = [statistics.median(r[i] for r in stage_runs) for i in range(8)]
    sort_ms = stage[7]

    # the plain form: binary32 model, one launch sequence for this array
    plain = None
    if not args.no_plain and precision != "fp32":
        pl = []
        for _ in range(2):
            job.copy_(pristine)
            torch.cuda.synchronize()
            st_p = nns.sort(job, None, model, precision="fp32", timing=True,
                            **tuned_sort_opts("fp32", n))
            pl.append(st_p["ms_stage"][7])
        plain = {"precision": "fp32", "sort_ms": min(pl), "job_ms": train_ms + min(pl),
                 "value": n / ((train_ms + min(pl)) / 1e3) / 1e6,
                 "sort_only_mkeys_s": n / (min(pl) / 1e3) / 1e6,
                 "sigma": st_p["sigma"], "trad_rate": st_p["trad_rate"],
                 "repaired": st_p["repaired"], "repair_ranges": st_p["repair_ranges"],
                 "oversized_buckets": st_p["oversized_buckets"],
                 "stage_ms": dict(zip(["predict", "partition", "bucket_bounds", "rounds",
                                       "finalize", "polish", "seam"], st_p["ms_stage"][:7]))}

    # the other tensor-core form, same model (slot resolution, conflicts, seam repairs, stage times)
    other = None
    if not args.no_plain and precision in ("bf16", "bf16x2"):
        op_ = "bf16" if precision == "bf16x2" else "bf16x2"
        oo = tuned_sort_opts(op_, n)
        runs = []
        for _ in range(2):
            job.copy_(pristine)
            torch.cuda.synchronize()
            runs.append(nns.sort(job, None, model, precision=op_, timing=True, **oo))
        best = min(runs, key=lambda r: r["ms_stage"][7])
        other = {"precision": op_, "sort_opts": oo, "sort_ms": best["ms_stage"][7],
                 "sigma": best["sigma"], "w_size": best["w_size"], "repaired": best["repaired"],
                 "repair_ranges": best["repair_ranges"],
                 "oversized_buckets": best["oversized_buckets"],
                 "stage_ms": dict(zip(["predict", "partition", "bucket_bounds", "rounds",
                                       "finalize", "polish", "seam"], best["ms_stage"][:7]))}

    # the compiled form of the same model: its piecewise-linear form evaluated per key by one binary
    # search and one multiply-add (the binary64 model's positions)
    compiled = None
    slot_error = None
    if not args.no_plain and precision != "pwl":
        po = tuned_sort_opts("pwl", n)
        runs = []
        for _ in range(2):
            job.copy_(pristine)
            torch.cuda.synchronize()
            runs.append(nns.sort(job, None, model, precision="pwl", timing=True, **po))
        best = min(runs, key=lambda r: r["ms_stage"][7])
        compiled = {"precision": "pwl", "sort_opts": po, "sort_ms": best["ms_stage"][7],
                    "job_ms": train_ms + best["ms_stage"][7],
                    "value": n / ((train_ms + best["ms_stage"][7]) / 1e3) / 1e6,
                    "sigma": best["sigma"], "repaired": best["repaired"],
                    "repair_ranges": best["repair_ranges"],
                    "oversized_buckets": best["oversized_buckets"],
                    "stage_ms": dict(zip(["predict", "partition", "bucket_bounds", "rounds",
                                          "finalize", "polish", "seam"], best["ms_stage"][:7]))}
        # slot displacement of each form against the binary64 model's positions, and the share of
        # keys that conflict in the first mapping round of its sort
        w1 = {precision: st["w_size"], "pwl": best["w_size"]}
        if plain is not None:
            w1["fp32"] = st_p["w_size"]
        if other is not None:
            w1[other["precision"]] = other["w_size"]
        ref, _ = nns.predict(pristine, model, precision="pwl", want_y=False)
        slot_error = {"against": "positions of the binary64 model (its compiled form)"}
        for p_ in ("bf16x2", "bf16", "fp32"):
            sp, _ = nns.predict(pristine, model, precision=p_, want_y=False)
            d = (sp - ref).abs_()
            slot_error[p_] = {"mean_abs": float(d.double().mean()), "max_abs": int(d.max()),
                              "frac_moved": float((d != 0).double().mean()),
                              "conflict_rate": (w1[p_][1] / n if p_ in w1 and len(w1[p_]) > 1
                                                else None)}
            del sp, d
        slot_error["pwl"] = {"conflict_rate": w1["pwl"][1] / n if len(w1["pwl"]) > 1 else None}
        del ref
        desc, params = model.describe()
        if desc["layers"] == 2 and pristine.dtype == torch.float32:
            slot_error["split_bf16_w2_rounding"] = w2_split_displacement(
                pristine[::max(1, n >> 18)].cpu().numpy(), desc, params, n * SORT["m"])

    # roofline of the dominant kernel stage: its mean duration over the timed steps (events the
    # library records on the call's stream)
    kb = 4
    arch_t = (ARCH["layers"], ARCH["h1"], ARCH["h2"])
    live = [statistics.mean(r[i] for r in timed_stages) for i in range(8)]
    dom = max(range(7), key=lambda i: live[i])
    roof = roofline_of(STAGES[dom], live[dom], n, kb, 0, precision, arch_t, st["partition_passes"], pk)
    roof["stage_share_of_sort"] = live[dom] / live[7]
    path = path_of(st, n, kb, 0, sort_ms, pk)

    # end to end through the host-array C entry point (pinned host buffers)
    e2e = None
    if rank == 0 or ws > 1:
        hbuf = torch.from_numpy(host.copy()).pin_memory()
        import ctypes as C
        to = nns._topts(**ARCH, **TRAIN)
        so = nns._sopts(sopts["m"], sopts["eps"], sopts["tau"], precision, sopts["bucket_log2"],
                        None, None, False, False, sopts["polish_blocks"])
        tt = []
        for k in range(max(2, min(args.steps, 3)) + 1):
            hbuf.numpy()[:] = host
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc = L.lib().nnsort_train_sort_host(C.c_void_p(hbuf.data_ptr()), None, n, 0, C.byref(to),
                                                C.byref(so), None, None, C.c_void_p(s.cuda_stream))
            t1 = time.perf_counter()
            L.check("nnsort_train_sort_host", rc)
            if k:
                tt.append(t1 - t0)
        e2e = {"value": n / statistics.median(tt) / 1e6, "unit": "Mkeys/s",
               "h2d_bytes_per_step": n * kb, "d2h_bytes_per_step": n * kb}

    # what the learned map gains on the headline input, then the other workloads
    del bufs
    abl = None
    if rank == 0 and not args.no_ablation:
        abl = {"headline input": ablation(nns, torch, pristine, model, n, kb, arch_t, None, 0,
                                          precision, pk)}
    del job
    configs = None
    if rank == 0 and not args.no_configs:
        del pristine
        torch.cuda.empty_cache()
        configs = {"1M uniform float32, 1-32-1 binary32": leg_c1(nns, W, torch, L, pk)}
        c3, c3_model, c3_src = leg_c3(nns, W, torch, L, pk)
        configs["64M uint64 key-value, 1-32-32-1"] = c3
        if abl is not None:
            abl["64M uint64 key-value input"] = ablation(nns, torch, c3_src, c3_model, c3_src.numel(),
                                                         8, (2, 32, 32), "u64", 3, c3["precision"], pk)
        del c3_model, c3_src
        torch.cuda.empty_cache()
        configs["4,096 float32 arrays, batched vs one call per array"] = leg_c4(nns, W, torch, L, pk)
        torch.cuda.empty_cache()

    serving = None
    if rank == 0 and not args.no_serve:
        serving = serving_leg(nns, W)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        ncpu = 300_000
        v, dt = oracle_job(ncpu)
        cpu = {"value": v, "unit": "Mkeys/s", "cores": 1, "kind": "oracle",
               "sample": f"{ncpu} keys of the same distribution, same model and recipe "
                         f"(1% sample, 100 full-batch binary64 steps), {dt:.1f} s",
               "host": cpu_info(), "library_sorts": cpu_sorts(host)}

    if rank == 0:
        line = {"metric": "Mkeys/s", "value": value, "unit": "Mkeys/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16" if precision in ("bf16", "bf16x2") else "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "n": n, "precision": precision,
                           "sort_opts": sopts,
                           "parallelism": "replicas" if ws > 1 else "single",
                           "l2": "inputs larger than L2 (each timed step sorts its own 1 GiB copy)"},
                "roofline": roof, "path": path,
                "breakdown_ms": {"train": train_ms, "sort": sort_ms,
                                 **{STAGES[i]: stage[i] for i in range(7)}},
                "sort_only_mkeys_s": n / (sort_ms / 1e3) / 1e6,
                "stats": {"rounds": st["t"], "w_size": st["w_size"], "sigma": st["sigma"],
                          "e": st["e"], "trad_rate": st["trad_rate"], "buckets": st["buckets"],
                          "oversized_buckets": st["oversized_buckets"], "repaired": st["repaired"],
                          "repair_ranges": st["repair_ranges"],
                          "final_train_loss": float(hist[-1])},
                "plain": plain, "other_tensor_form": other, "compiled_form": compiled,
                "slot_error": slot_error, "ablation": abl, "configs": configs,
                "serving": serving, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk.summary(),
                "gpu_launches": int(launches)}
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
