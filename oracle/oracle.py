"""numpy front end of the plain C oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's CPU-baseline leg
are the only callers. It never touches the CUDA library and the CUDA library never touches it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

F32, F64, U32, U64 = 0, 1, 2, 3
ORDBITS, VALUE = 0, 1
MSE, HUBER = 0, 1
MAX_ROUNDS = 8

_DT = {np.dtype(np.float32): F32, np.dtype(np.float64): F64,
       np.dtype(np.uint32): U32, np.dtype(np.uint64): U64}


_CPU_SRC = os.path.join(_HERE, "cpu_sorts.cpp")
_CPU_LIB = os.path.join(_HERE, "libcpusorts.so")


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no FMA contraction, so binary32 steps are the written ones)
    and the library CPU sorts the benchmark times as a baseline (libcpusorts.so, g++)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-fno-fast-math", "-o", _LIB, _SRC, "-lm"])
    if force or not os.path.exists(_CPU_LIB) or os.path.getmtime(_CPU_LIB) < os.path.getmtime(_CPU_SRC):
        subprocess.check_call(["g++", "-O3", "-std=c++17", "-fPIC", "-shared", "-pthread", "-o",
                               _CPU_LIB, _CPU_SRC])
    return _LIB


def cpu_sort(keys: np.ndarray, algo: str, threads: int = 1):
    """(sorted copy, seconds) of a library CPU sort: 'stable_sort' / 'sort' (std::, one thread) or
    'parallel' (std::sort of per-thread chunks + parallel pairwise std::merge over `threads`)."""
    build()
    lib_ = C.CDLL(_CPU_LIB)
    lib_.cpu_sort.restype = C.c_double
    lib_.cpu_sort.argtypes = [C.c_void_p, C.c_int, C.c_uint64, C.c_void_p, C.c_int, C.c_int]
    keys = np.ascontiguousarray(keys)
    out = np.empty_like(keys)
    code = {np.dtype(np.float32): 0, np.dtype(np.float64): 1, np.dtype(np.uint64): 3}[keys.dtype]
    dt = lib_.cpu_sort(_p(keys), code, keys.shape[0], _p(out),
                       {"stable_sort": 0, "sort": 1, "parallel": 2}[algo], threads)
    return out, float(dt)


class Norm(C.Structure):
    _fields_ = [("dtype", C.c_int32), ("translate", C.c_int32), ("lo_bits", C.c_uint64),
                ("lo_val", C.c_double), ("scale", C.c_double), ("lo_f", C.c_float),
                ("scale_f", C.c_float)]


class Arch(C.Structure):
    _fields_ = [("layers", C.c_int32), ("h1", C.c_int32), ("h2", C.c_int32)]


class TrainOpts(C.Structure):
    _fields_ = [("arch", Arch), ("translate", C.c_int32), ("loss", C.c_int32),
                ("huber_delta", C.c_double), ("sample_n", C.c_uint64), ("steps", C.c_uint64),
                ("batch", C.c_uint64), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("adam_eps", C.c_double), ("seed", C.c_uint64),
                ("monotone", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("t", C.c_uint32), ("eps", C.c_uint32), ("n", C.c_uint64), ("L", C.c_uint64),
                ("tau", C.c_uint64), ("w_size", C.c_uint64 * (MAX_ROUNDS + 1)),
                ("placed", C.c_uint64 * MAX_ROUNDS), ("out_of_order", C.c_uint64 * MAX_ROUNDS)]

    def as_dict(self) -> dict:
        t = self.t
        return {"t": t, "eps": self.eps, "n": self.n, "L": self.L, "tau": self.tau,
                "w_size": [self.w_size[i] for i in range(t + 1)],
                "placed": [self.placed[i] for i in range(t)],
                "out_of_order": [self.out_of_order[i] for i in range(t)]}


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.c_void_p
        u64, i32, f32, f64 = C.c_uint64, C.c_int, C.c_float, C.c_double
        sig = {
            "orc_mix64": (u64, [u64]),
            "orc_rng": (u64, [u64, u64]),
            "orc_stream_seed": (u64, [u64, u64]),
            "orc_ordbits": (u64, [P, i32, u64]),
            "orc_translate_f32": (None, [P, i32, u64, P, P]),
            "orc_translate_f64": (None, [P, i32, u64, P, P]),
            "orc_make_norm": (None, [P, i32, P, u64, i32, P]),
            "orc_num_params": (u64, [P]),
            "orc_mlp_forward_f32": (None, [P, P, P, u64, P]),
            "orc_mlp_layer1_f32": (None, [P, P, P, u64, P]),
            "orc_mlp_forward_f64": (None, [P, P, P, u64, P]),
            "orc_mlp_loss_grad_f64": (f64, [P, P, P, P, u64, i32, f64, P, P]),
            "orc_adam_f64": (None, [P, P, P, P, u64, u64, f64, f64, f64, f64]),
            "orc_init_params": (None, [P, u64, P]),
            "orc_sample_labels": (i32, [P, i32, u64, u64, u64, i32, P, P, P, P]),
            "orc_train": (i32, [P, i32, u64, P, P, P, P]),
            "orc_nm_split": (None, [u64, f32, P, P, P]),
            "orc_slot1": (C.c_uint32, [f32, f32, f32, u64]),
            "orc_predict_slots": (i32, [P, i32, u64, P, P, P, f32, P, P]),
            "orc_sort_rows": (None, [P, i32, P, u64]),
            "orc_nnsort": (i32, [P, i32, P, u64, P, u64, i32, u64, P, P, P, P]),
            "orc_nnsort_model": (i32, [P, i32, P, u64, P, P, P, f32, i32, u64, P, P, P, P]),
            "orc_stable_sort": (None, [P, i32, P, u64, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def dtype_code(a: np.ndarray) -> int:
    return _DT[a.dtype]


# ------------------------------------------------------------------------------------------
@dataclass
class Model:
    """Oracle-side model f: architecture, normaliser and binary32 parameters."""
    layers: int
    h1: int
    h2: int
    norm: Norm
    params: np.ndarray  # float32

    @property
    def arch(self) -> Arch:
        return Arch(self.layers, self.h1, self.h2)


def num_params(layers: int, h1: int, h2: int = 0) -> int:
    return int(lib().orc_num_params(C.byref(Arch(layers, h1, h2))))


def rng(seed: int, i: int) -> int:
    return int(lib().orc_rng(seed, i))


def ordbits(keys: np.ndarray) -> np.ndarray:
    keys = np.ascontiguousarray(keys)
    dt = dtype_code(keys)
    return np.array([lib().orc_ordbits(_p(keys), dt, i) for i in range(keys.shape[0])],
                    dtype=np.uint64)


def make_norm(keys: np.ndarray, rows: np.ndarray, translate: int) -> Norm:
    keys = np.ascontiguousarray(keys)
    rows = np.ascontiguousarray(rows, dtype=np.uint64)
    nm = Norm()
    lib().orc_make_norm(_p(keys), dtype_code(keys), _p(rows), rows.shape[0], translate, C.byref(nm))
    return nm


def translate_f32(keys: np.ndarray, nm: Norm) -> np.ndarray:
    keys = np.ascontiguousarray(keys)
    x = np.empty(keys.shape[0], dtype=np.float32)
    lib().orc_translate_f32(_p(keys), dtype_code(keys), keys.shape[0], C.byref(nm), _p(x))
    return x


def translate_f64(keys: np.ndarray, nm: Norm) -> np.ndarray:
    keys = np.ascontiguousarray(keys)
    x = np.empty(keys.shape[0], dtype=np.float64)
    lib().orc_translate_f64(_p(keys), dtype_code(keys), keys.shape[0], C.byref(nm), _p(x))
    return x


def mlp_forward_f32(layers, h1, h2, params, x) -> np.ndarray:
    params = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    y = np.empty_like(x)
    lib().orc_mlp_forward_f32(C.byref(Arch(layers, h1, h2)), _p(params), _p(x), x.shape[0], _p(y))
    return y


def mlp_layer1_f32(layers, h1, h2, params, x) -> np.ndarray:
    params = np.ascontiguousarray(params, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    h = np.empty((x.shape[0], h1), dtype=np.float32)
    lib().orc_mlp_layer1_f32(C.byref(Arch(layers, h1, h2)), _p(params), _p(x), x.shape[0], _p(h))
    return h


def mlp_forward_f64(layers, h1, h2, params, x) -> np.ndarray:
    params = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    lib().orc_mlp_forward_f64(C.byref(Arch(layers, h1, h2)), _p(params), _p(x), x.shape[0], _p(y))
    return y


def mlp_loss_grad_f64(layers, h1, h2, params, x, label, loss=MSE, delta=0.01):
    params = np.ascontiguousarray(params, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    label = np.ascontiguousarray(label, dtype=np.float64)
    g = np.empty_like(params)
    gx = np.empty_like(x)
    L = lib().orc_mlp_loss_grad_f64(C.byref(Arch(layers, h1, h2)), _p(params), _p(x), _p(label),
                                     x.shape[0], loss, delta, _p(g), _p(gx))
    return float(L), g, gx


def adam_f64(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_adam_f64(_p(p), _p(g), _p(m), _p(v), p.shape[0], step, lr, b1, b2, eps)


def init_params(layers, h1, h2, seed) -> np.ndarray:
    p = np.empty(num_params(layers, h1, h2), dtype=np.float32)
    lib().orc_init_params(C.byref(Arch(layers, h1, h2)), seed, _p(p))
    return p


def sample_labels(keys: np.ndarray, S: int, seed: int, translate: int = ORDBITS):
    keys = np.ascontiguousarray(keys)
    rows = np.empty(S, dtype=np.uint64)
    x = np.empty(S, dtype=np.float32)
    lab = np.empty(S, dtype=np.float32)
    nm = Norm()
    rc = lib().orc_sample_labels(_p(keys), dtype_code(keys), keys.shape[0], S, seed, translate,
                                 _p(rows), C.byref(nm), _p(x), _p(lab))
    if rc != 0:
        raise ValueError("orc_sample_labels failed (NaN key or empty input)")
    return rows, nm, x, lab


def train(keys: np.ndarray, layers=1, h1=32, h2=0, translate=ORDBITS, loss=MSE, huber_delta=0.01,
          sample_n=10_000, steps=100, batch=0, lr=1e-2, beta1=0.9, beta2=0.999, adam_eps=1e-8,
          seed=0, monotone=False):
    """Binary64 training; returns (Model with params rounded to binary32, params f64, loss history)."""
    keys = np.ascontiguousarray(keys)
    o = TrainOpts(Arch(layers, h1, h2), translate, loss, huber_delta, sample_n, steps, batch, lr,
                  beta1, beta2, adam_eps, seed, 1 if monotone else 0)
    P = num_params(layers, h1, h2)
    p = np.empty(P, dtype=np.float64)
    hist = np.empty(max(steps, 1), dtype=np.float64)
    nm = Norm()
    rc = lib().orc_train(_p(keys), dtype_code(keys), keys.shape[0], C.byref(o), C.byref(nm), _p(p),
                         _p(hist))
    if rc != 0:
        raise ValueError("orc_train failed")
    return Model(layers, h1, h2, nm, p.astype(np.float32)), p, hist[:steps]


def nm_split(n: int, m: float = 1.25):
    L = C.c_uint64()
    hi = C.c_float()
    lo = C.c_float()
    lib().orc_nm_split(n, m, C.byref(L), C.byref(hi), C.byref(lo))
    return int(L.value), float(hi.value), float(lo.value)


def slot1(y: float, nm_hi: float, nm_lo: float, L: int) -> int:
    return int(lib().orc_slot1(y, nm_hi, nm_lo, L))


def predict_slots(keys: np.ndarray, model: Model, m: float = 1.25):
    keys = np.ascontiguousarray(keys)
    n = keys.shape[0]
    slots = np.empty(n, dtype=np.uint32)
    y = np.empty(n, dtype=np.float32)
    params = np.ascontiguousarray(model.params, dtype=np.float32)
    rc = lib().orc_predict_slots(_p(keys), dtype_code(keys), n, C.byref(model.norm),
                                 C.byref(model.arch), _p(params), m, _p(slots), _p(y))
    if rc != 0:
        raise ValueError("NaN key")
    return slots, y


def nnsort(keys: np.ndarray, slots: np.ndarray, L: int, eps: int = 3, tau: int = 1024,
           payload: np.ndarray | None = None, want_fate: bool = False):
    """Sequential NN-sort given each key's slot. Returns (sorted keys, sorted payload or None,
    stats dict, fate or None)."""
    keys = np.ascontiguousarray(keys)
    slots = np.ascontiguousarray(slots, dtype=np.uint32)
    n = keys.shape[0]
    out = np.empty_like(keys)
    outp = None
    if payload is not None:
        payload = np.ascontiguousarray(payload, dtype=np.int32)
        outp = np.empty_like(payload)
    fate = np.empty(n, dtype=np.int8) if want_fate else None
    st = Stats()
    rc = lib().orc_nnsort(_p(keys), dtype_code(keys), _p(payload), n, _p(slots), L, eps, tau,
                          _p(out), _p(outp), C.byref(st), _p(fate))
    if rc != 0:
        raise ValueError(f"orc_nnsort failed ({rc})")
    return out, outp, st.as_dict(), fate


def nnsort_model(keys: np.ndarray, model: Model, m: float = 1.25, eps: int = 3, tau: int = 1024,
                 payload: np.ndarray | None = None, want_fate: bool = False):
    keys = np.ascontiguousarray(keys)
    n = keys.shape[0]
    out = np.empty_like(keys)
    outp = None
    if payload is not None:
        payload = np.ascontiguousarray(payload, dtype=np.int32)
        outp = np.empty_like(payload)
    fate = np.empty(n, dtype=np.int8) if want_fate else None
    st = Stats()
    params = np.ascontiguousarray(model.params, dtype=np.float32)
    rc = lib().orc_nnsort_model(_p(keys), dtype_code(keys), _p(payload), n, C.byref(model.norm),
                                C.byref(model.arch), _p(params), m, eps, tau, _p(out), _p(outp),
                                C.byref(st), _p(fate))
    if rc != 0:
        raise ValueError(f"orc_nnsort_model failed ({rc})")
    return out, outp, st.as_dict(), fate


def stable_sort(keys: np.ndarray, payload: np.ndarray | None = None):
    keys = np.ascontiguousarray(keys)
    out = np.empty_like(keys)
    outp = None
    if payload is not None:
        payload = np.ascontiguousarray(payload, dtype=np.int32)
        outp = np.empty_like(payload)
    lib().orc_stable_sort(_p(keys), dtype_code(keys), _p(payload), keys.shape[0], _p(out), _p(outp))
    return out, outp
