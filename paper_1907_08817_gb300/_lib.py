"""ctypes declarations of libnnsort.so's C ABI (include/nnsort.h). Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnnsort.so")

MAX_ROUNDS = 8
F32, F64, U32, U64 = 0, 1, 2, 3
ORDBITS, VALUE = 0, 1
PREC_FP32, PREC_BF16, PREC_BF16X2, PREC_PWL = 0, 1, 2, 3
LOSS_MSE, LOSS_HUBER = 0, 1

STATUS = {0: "ok", -1: "invalid argument", -2: "NaN key", -3: "out of memory",
          -4: "over the HBM budget", -5: "CUDA error", -6: "device wait timed out",
          -7: "unsupported option", -8: "invalid state"}


class ModelDesc(C.Structure):
    _fields_ = [("dtype", C.c_int32), ("translate", C.c_int32), ("layers", C.c_int32),
                ("h1", C.c_int32), ("h2", C.c_int32), ("lo_bits", C.c_uint64),
                ("lo_val", C.c_double), ("scale", C.c_double)]


class TrainOpts(C.Structure):
    _fields_ = [("layers", C.c_int32), ("h1", C.c_int32), ("h2", C.c_int32),
                ("translate", C.c_int32), ("loss", C.c_int32), ("huber_delta", C.c_float),
                ("sample_n", C.c_uint64), ("steps", C.c_uint32), ("batch", C.c_uint32),
                ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("adam_eps", C.c_float), ("seed", C.c_uint64), ("monotone", C.c_int32)]


class SortOpts(C.Structure):
    _fields_ = [("m", C.c_float), ("eps", C.c_int32), ("tau", C.c_uint64),
                ("precision", C.c_int32), ("bucket_log2", C.c_int32),
                ("d_slots", C.c_void_p), ("d_fate", C.c_void_p), ("no_sync", C.c_int32),
                ("timing", C.c_int32), ("polish_blocks", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("rounds", C.c_uint32), ("eps", C.c_uint32), ("n", C.c_uint64),
                ("L", C.c_uint64), ("tau", C.c_uint64),
                ("w_size", C.c_uint64 * (MAX_ROUNDS + 1)),
                ("placed", C.c_uint64 * MAX_ROUNDS),
                ("out_of_order", C.c_uint64 * MAX_ROUNDS),
                ("sigma", C.c_double * MAX_ROUNDS), ("e", C.c_double * MAX_ROUNDS),
                ("trad_rate", C.c_double), ("buckets", C.c_uint64),
                ("oversized_buckets", C.c_uint64), ("repaired", C.c_uint64),
                ("ms_stage", C.c_float * 8), ("partition_passes", C.c_uint32),
                ("bucket_log2", C.c_uint32), ("repair_ranges", C.c_uint64)]

    def as_dict(self) -> dict:
        t = self.rounds
        return {"t": t, "eps": self.eps, "n": self.n, "L": self.L, "tau": self.tau,
                "w_size": [self.w_size[i] for i in range(t + 1)],
                "placed": [self.placed[i] for i in range(t)],
                "out_of_order": [self.out_of_order[i] for i in range(t)],
                "sigma": [self.sigma[i] for i in range(t)],
                "e": [self.e[i] for i in range(t)], "trad_rate": self.trad_rate,
                "buckets": self.buckets, "oversized_buckets": self.oversized_buckets,
                "repaired": self.repaired, "ms_stage": [self.ms_stage[i] for i in range(8)],
                "partition_passes": self.partition_passes, "bucket_log2": self.bucket_log2,
                "repair_ranges": self.repair_ranges}


class NNSortError(RuntimeError):
    def __init__(self, fn: str, status: int, cuda: int = 0):
        msg = f"{fn}: {STATUS.get(status, status)}"
        if status == -5:
            msg += f" (cudaError {cuda})"
        super().__init__(msg)
        self.status = status


_lib = None


def lib():
    """Loads libnnsort.so; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libnnsort.so is missing at {LIB_PATH}: run "
                           "`python -c 'import __graft_entry__ as g; g.build()'` first")
    L = C.CDLL(LIB_PATH)
    P, u64, i32, f32, sz = C.c_void_p, C.c_uint64, C.c_int32, C.c_float, C.c_size_t
    sig = {
        "nnsort_version": (C.c_int, []),
        "nnsort_strerror": (C.c_char_p, [C.c_int]),
        "nnsort_last_cuda_error": (C.c_int, []),
        "nnsort_default_train_opts": (None, [P]),
        "nnsort_default_sort_opts": (None, [P]),
        "nnsort_release": (C.c_int, []),
        "nnsort_stream_status": (C.c_int, [P]),
        "nnsort_selftest_wait": (C.c_int, [C.c_uint32, P]),
        "nnsort_workspace_bytes": (sz, [u64, i32, i32, P]),
        "nnsort_model_create": (C.c_int, [P, P, P]),
        "nnsort_model_free": (C.c_int, [P]),
        "nnsort_model_describe": (C.c_int, [P, P, P]),
        "nnsort_model_blob_size": (sz, [P]),
        "nnsort_model_save": (C.c_int, [P, P, sz]),
        "nnsort_model_load": (C.c_int, [P, sz, P]),
        "nnsort_mlp_pwl": (C.c_int, [i32, i32, i32, P, P, P, P, C.c_uint32, P]),
        "nnsort_sample_labels": (C.c_int, [P, u64, i32, u64, u64, i32, P, P, P, P, P]),
        "nnsort_train": (C.c_int, [P, u64, i32, P, P, P, P]),
        "nnsort_mlp_forward": (C.c_int, [P, i32, i32, i32, P, u64, P, P]),
        "nnsort_mlp_backward": (C.c_int, [P, i32, i32, i32, P, P, u64, P, P, P]),
        "nnsort_mlp_loss_grad": (C.c_int, [P, i32, i32, i32, P, P, u64, i32, f32, P, P, P]),
        "nnsort_predict": (C.c_int, [P, u64, i32, P, f32, i32, P, P, P]),
        "nnsort_sort": (C.c_int, [P, P, u64, i32, P, P, P, P]),
        "nnsort_sort_host": (C.c_int, [P, P, u64, i32, P, P, P, P]),
        "nnsort_sort_batch": (C.c_int, [P, P, P, i32, i32, P, P, P, P]),
        "nnsort_train_sort_host": (C.c_int, [P, P, u64, i32, P, P, P, P, P]),
        "nnsort_launch_count": (u64, []),
        "nnsort_sort_noalloc": (C.c_int, [P, P, u64, i32, P, P, P, P]),
        "nnsort_radix_sort": (C.c_int, [P, P, u64, i32, P]),
        "nnsort_train_batch": (C.c_int, [P, P, i32, i32, P, P, P, P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(fn: str, rc: int) -> None:
    if rc != 0:
        raise NNSortError(fn, rc, lib().nnsort_last_cuda_error())


def exported_symbols() -> list[str]:
    """Every entry point name the binding declares (the header's declarations)."""
    return ["nnsort_version", "nnsort_strerror", "nnsort_last_cuda_error",
            "nnsort_default_train_opts", "nnsort_default_sort_opts", "nnsort_release",
            "nnsort_stream_status", "nnsort_selftest_wait", "nnsort_workspace_bytes",
            "nnsort_model_create",
            "nnsort_model_free", "nnsort_model_describe", "nnsort_model_blob_size",
            "nnsort_model_save", "nnsort_model_load", "nnsort_mlp_pwl", "nnsort_sample_labels",
            "nnsort_train",
            "nnsort_mlp_forward", "nnsort_mlp_backward", "nnsort_mlp_loss_grad",
            "nnsort_predict", "nnsort_sort", "nnsort_sort_host", "nnsort_sort_batch",
            "nnsort_train_sort_host", "nnsort_launch_count", "nnsort_sort_noalloc", "nnsort_radix_sort", "nnsort_train_batch",
            "nnsort_default_server_opts", "nnsort_server_create", "nnsort_server_submit",
            "nnsort_server_poll", "nnsort_server_wait", "nnsort_server_destroy"]


class ServerOpts(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("workers", C.c_int32), ("max_batch", C.c_int32),
                ("max_batch_keys", C.c_uint64), ("train", TrainOpts), ("sort", SortOpts)]


PENDING = 1
SERVER_SIGS = {
    "nnsort_default_server_opts": (None, [C.c_void_p]),
    "nnsort_server_create": (C.c_int, [C.c_void_p, C.c_void_p]),
    "nnsort_server_submit": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_uint64, C.c_int32,
                                       C.c_uint64, C.c_void_p]),
    "nnsort_server_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]),
    "nnsort_server_wait": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p]),
    "nnsort_server_destroy": (C.c_int, [C.c_void_p]),
}


def server_lib():
    L = lib()
    for name, (res, args) in SERVER_SIGS.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L
