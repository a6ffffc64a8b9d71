"""GB300-native NN-sort (arXiv 1907.08817): Python binding of libnnsort.so.

Every step of the method runs in the library's CUDA kernels; this module only marshals torch
tensors (device memory, streams) into the C ABI declared in include/nnsort.h. If the library has
not been built, every call raises -- there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _lib as L
from ._lib import (F32, F64, U32, U64, ORDBITS, VALUE, PREC_BF16, PREC_FP32, LOSS_HUBER,
                   LOSS_MSE, NNSortError)

__all__ = ["Model", "train", "train_batch", "sample_labels", "predict", "sort", "sort_batch", "sort_host", "radix_sort",
           "mlp_forward", "mlp_backward", "mlp_loss_grad", "NNSortMLPFunction", "NNSortError",
           "key_code", "release", "workspace_bytes", "stream_status", "version"]


def _torch():
    import torch
    return torch


def version() -> int:
    return int(L.lib().nnsort_version())


def release() -> None:
    L.check("nnsort_release", L.lib().nnsort_release())


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def stream_status(stream=None) -> int:
    return int(L.lib().nnsort_stream_status(_stream(stream)))


def selftest_wait(limit_us: int = 1000, stream=None) -> int:
    """Runs the library's bounded device-side wait on a flag that nothing sets; the status is
    NNSORT_E_TIMEOUT (-6) when the wait expired as it must."""
    return int(L.lib().nnsort_selftest_wait(int(limit_us), _stream(stream)))


def key_code(t, key_type: str | None = None) -> int:
    """nnsort_dtype of a key tensor/array. int32/int64 storage holds unsigned keys' bits and needs
    key_type='u32'/'u64'."""
    if key_type is not None:
        return {"f32": F32, "f64": F64, "u32": U32, "u64": U64}[key_type]
    name = str(t.dtype).replace("torch.", "")
    m = {"float32": F32, "float64": F64, "uint32": U32, "uint64": U64}
    if name not in m:
        raise TypeError(f"key dtype {t.dtype} needs key_type= ('u32' or 'u64' for integer bits)")
    return m[name]


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _prec(p) -> int:
    if isinstance(p, int):
        return p
    return {"fp32": PREC_FP32, "bf16": PREC_BF16, "bf16x2": L.PREC_BF16X2, "pwl": L.PREC_PWL}[p]


def _tr(t) -> int:
    if isinstance(t, int):
        return t
    return {"ordbits": ORDBITS, "value": VALUE}[t]


# ------------------------------------------------------------------------------------ model f
@dataclass
class _Handle:
    ptr: C.c_void_p


class Model:
    """Opaque device-resident model (ReLU MLP + normaliser of translate(A))."""

    def __init__(self, handle: C.c_void_p):
        self._h = handle

    @property
    def handle(self) -> C.c_void_p:
        return self._h

    @property
    def shape(self) -> tuple:
        """(layers, h1, h2) of the MLP."""
        if getattr(self, "_shape", None) is None:
            d = L.ModelDesc()
            L.check("nnsort_model_describe", L.lib().nnsort_model_describe(self._h, C.byref(d), None))
            self._shape = (d.layers, d.h1, d.h2)
        return self._shape

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and L._lib is not None:
            L._lib.nnsort_model_free(h)
            self._h = None

    @classmethod
    def create(cls, dtype: int, layers: int, h1: int, h2: int, params, translate=ORDBITS,
               lo_bits: int = 0, lo_val: float = 0.0, scale: float = 1.0) -> "Model":
        d = L.ModelDesc(dtype, _tr(translate), layers, h1, h2, lo_bits, lo_val, scale)
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        h = C.c_void_p()
        L.check("nnsort_model_create", L.lib().nnsort_model_create(
            C.byref(d), p.ctypes.data_as(C.c_void_p), C.byref(h)))
        return cls(h)

    def describe(self):
        d = L.ModelDesc()
        L.check("nnsort_model_describe", L.lib().nnsort_model_describe(self._h, C.byref(d), None))
        P = (3 * d.h1 + 1) if d.layers == 1 else (2 * d.h1 + d.h2 * d.h1 + 2 * d.h2 + 1)
        p = np.empty(P, dtype=np.float32)
        L.check("nnsort_model_describe", L.lib().nnsort_model_describe(
            self._h, None, p.ctypes.data_as(C.c_void_p)))
        return {"dtype": d.dtype, "translate": d.translate, "layers": d.layers, "h1": d.h1,
                "h2": d.h2, "lo_bits": d.lo_bits, "lo_val": d.lo_val, "scale": d.scale}, p

    def pwl(self):
        """The piecewise-linear form of f: see mlp_pwl."""
        d, p = self.describe()
        return mlp_pwl(p, d["layers"], d["h1"], d["h2"])

    def save(self) -> bytes:
        n = L.lib().nnsort_model_blob_size(self._h)
        buf = (C.c_char * n)()
        L.check("nnsort_model_save", L.lib().nnsort_model_save(self._h, buf, n))
        return bytes(buf)

    @classmethod
    def load(cls, blob: bytes) -> "Model":
        h = C.c_void_p()
        b = C.create_string_buffer(blob, len(blob))
        L.check("nnsort_model_load", L.lib().nnsort_model_load(b, len(blob), C.byref(h)))
        return cls(h)


def _topts(**kw) -> L.TrainOpts:
    o = L.TrainOpts()
    L.lib().nnsort_default_train_opts(C.byref(o))
    for k, v in kw.items():
        if v is None:
            continue
        if k == "translate":
            v = _tr(v)
        if k == "loss":
            v = {"mse": LOSS_MSE, "huber": LOSS_HUBER}.get(v, v)
        setattr(o, k, v)
    return o


def train(keys, *, key_type=None, layers=1, h1=32, h2=0, translate="ordbits", loss="mse",
          huber_delta=0.01, sample_n=10_000, steps=100, batch=0, lr=1e-2, beta1=0.9, beta2=0.999,
          adam_eps=1e-8, seed=0, monotone=False, stream=None):
    """Trains f on the device from a seeded sample of `keys` (device tensor). Returns
    (Model, per-step loss history as numpy)."""
    o = _topts(layers=layers, h1=h1, h2=h2, translate=translate, loss=loss,
               huber_delta=huber_delta, sample_n=sample_n, steps=steps, batch=batch, lr=lr,
               beta1=beta1, beta2=beta2, adam_eps=adam_eps, seed=seed,
               monotone=1 if monotone else 0)
    hist = np.zeros(max(steps, 1), dtype=np.float32)
    h = C.c_void_p()
    L.check("nnsort_train", L.lib().nnsort_train(
        _ptr(keys), keys.numel(), key_code(keys, key_type), C.byref(o), C.byref(h),
        hist.ctypes.data_as(C.c_void_p), _stream(stream)))
    return Model(h), hist[:steps]


def train_batch(keys_list, *, sample_ns=None, key_type=None, layers=1, h1=16, h2=0,
                translate="ordbits", loss="mse", huber_delta=0.01, sample_n=10_000, steps=100,
                batch=0, lr=1e-2, beta1=0.9, beta2=0.999, adam_eps=1e-8, seed=0, stream=None):
    """Trains one model per array of keys_list in one pass (nnsort_train_batch): model j from its
    own seeded sample (sample_ns[j] keys, or sample_n) with seed seed + j. Returns (models, losses
    as a count x steps numpy array)."""
    cnt = len(keys_list)
    o = _topts(layers=layers, h1=h1, h2=h2, translate=translate, loss=loss,
               huber_delta=huber_delta, sample_n=sample_n, steps=steps, batch=batch, lr=lr,
               beta1=beta1, beta2=beta2, adam_eps=adam_eps, seed=seed, monotone=0)
    kp = (C.c_void_p * cnt)(*[k.data_ptr() for k in keys_list])
    ns = (C.c_uint64 * cnt)(*[k.numel() for k in keys_list])
    sp = None if sample_ns is None else (C.c_uint64 * cnt)(*[int(v) for v in sample_ns])
    hs = (C.c_void_p * cnt)()
    hist = np.zeros((cnt, max(steps, 1)), dtype=np.float32)
    code = key_code(keys_list[0], key_type) if cnt else F32
    L.check("nnsort_train_batch", L.lib().nnsort_train_batch(
        kp, ns, cnt, code, C.byref(o), sp, hs, hist.ctypes.data_as(C.c_void_p), _stream(stream)))
    return [Model(C.c_void_p(h)) for h in hs], hist[:, :steps]


def sample_labels(keys, S: int, seed: int = 0, translate="ordbits", key_type=None, stream=None):
    """Training data of Sec. "Training": (x, label, rows) device tensors and the normaliser."""
    torch = _torch()
    x = torch.empty(S, dtype=torch.float32, device=keys.device)
    lab = torch.empty(S, dtype=torch.float32, device=keys.device)
    rows = torch.empty(S, dtype=torch.int32, device=keys.device)
    d = L.ModelDesc()
    L.check("nnsort_sample_labels", L.lib().nnsort_sample_labels(
        _ptr(keys), keys.numel(), key_code(keys, key_type), S, seed, _tr(translate), C.byref(d),
        _ptr(x), _ptr(lab), _ptr(rows), _stream(stream)))
    norm = {"dtype": d.dtype, "translate": d.translate, "lo_bits": d.lo_bits,
            "lo_val": d.lo_val, "scale": d.scale}
    return x, lab, rows, norm


def predict(keys, model: Model, m: float = 1.25, precision="fp32", key_type=None, stream=None,
            want_y: bool = True):
    """Positions round(f(x) n m) (int64 tensor) and F(x) (float32 tensor or None)."""
    torch = _torch()
    n = keys.numel()
    slots = torch.empty(n, dtype=torch.int32, device=keys.device)
    y = torch.empty(n, dtype=torch.float32, device=keys.device) if want_y else None
    L.check("nnsort_predict", L.lib().nnsort_predict(
        _ptr(keys), n, key_code(keys, key_type), model.handle, m, _prec(precision), _ptr(slots),
        _ptr(y), _stream(stream)))
    return slots.to(torch.int64) & 0xFFFFFFFF, y


def _sopts(m, eps, tau, precision, bucket_log2, slots, fate, no_sync, timing=False,
           polish_blocks=0) -> L.SortOpts:
    o = L.SortOpts()
    L.lib().nnsort_default_sort_opts(C.byref(o))
    o.m, o.eps, o.tau, o.precision, o.bucket_log2 = m, eps, tau, _prec(precision), bucket_log2
    o.timing = 1 if timing else 0
    o.polish_blocks = polish_blocks
    o.d_slots = None if slots is None else slots.data_ptr()
    o.d_fate = None if fate is None else fate.data_ptr()
    o.no_sync = 1 if no_sync else 0
    return o


def _tuned(model, n, dtype, precision, eps, bucket_log2, polish_blocks):
    """Fills the parameters left to the library (bucket_log2=0, polish_blocks=0, eps='auto') from
    the autotuner's table for this key type, size class, model shape and precision."""
    if model is None or (bucket_log2 and polish_blocks and eps != "auto"):
        return (3 if eps == "auto" else eps), bucket_log2, polish_blocks
    from . import autotune
    t = autotune.tuned_options(dtype, n, *model.shape, precision)
    return (t["eps"] if eps == "auto" else eps, bucket_log2 or t["bucket_log2"],
            polish_blocks or t["polish_blocks"])


def sort(keys, payload=None, model: Model | None = None, *, m=1.25, eps=3, tau=1024,
         precision="fp32", bucket_log2=0, slots=None, fate: bool = False, stats: bool = True,
         timing: bool = False, polish_blocks: int = 0, key_type=None, stream=None):
    """NN-sort in place. `slots` (int32 device tensor of positions) replaces the model.
    bucket_log2=0 / polish_blocks=0 / eps='auto' take the autotuned setting for this workload
    class (the library's defaults where none was tuned).
    Returns the stats dict (or None), plus the per-row fate tensor when fate=True."""
    torch = _torch()
    n = keys.numel()
    eps, bucket_log2, polish_blocks = _tuned(None if slots is not None else model, n,
                                             key_code(keys, key_type), precision, eps,
                                             bucket_log2, polish_blocks)
    ft = torch.zeros(n, dtype=torch.int8, device=keys.device) if fate else None
    o = _sopts(m, eps, tau, precision, bucket_log2, slots, ft, not stats, timing, polish_blocks)
    st = L.Stats() if (stats or timing) else None
    rc = L.lib().nnsort_sort(_ptr(keys), _ptr(payload), n, key_code(keys, key_type),
                             None if model is None else model.handle, C.byref(o),
                             None if st is None else C.byref(st), _stream(stream))
    L.check("nnsort_sort", rc)
    out = st.as_dict() if st is not None else None
    return (out, ft) if fate else out


def radix_sort(keys, payload=None, *, key_type=None, stream=None) -> None:
    """The "no model" reference: stable LSD radix sort of the keys (and payload) in place, every
    pass the pipeline's partition kernel (nnsort_radix_sort)."""
    L.check("nnsort_radix_sort", L.lib().nnsort_radix_sort(
        _ptr(keys), _ptr(payload), keys.numel(), key_code(keys, key_type), _stream(stream)))


def sort_host(keys: np.ndarray, payload: np.ndarray | None = None, model: Model | None = None, *,
              m=1.25, eps=3, tau=1024, precision="fp32", bucket_log2=0, stream=None):
    """End-to-end sort of host arrays in place (copies in and out inside the library)."""
    assert keys.flags.c_contiguous
    code = {np.dtype(np.float32): F32, np.dtype(np.float64): F64, np.dtype(np.uint32): U32,
            np.dtype(np.uint64): U64}[keys.dtype]
    o = _sopts(m, eps, tau, precision, bucket_log2, None, None, False)
    st = L.Stats()
    pp = None
    if payload is not None:
        assert payload.dtype == np.int32 and payload.flags.c_contiguous
        pp = payload.ctypes.data_as(C.c_void_p)
    L.check("nnsort_sort_host", L.lib().nnsort_sort_host(
        keys.ctypes.data_as(C.c_void_p), pp, keys.shape[0], code,
        None if model is None else model.handle, C.byref(o), C.byref(st), _stream(stream)))
    return st.as_dict()


def sort_batch(keys_list, models, payloads=None, *, m=1.25, eps=3, tau=1024, precision="fp32",
               bucket_log2=0, polish_blocks=0, stats=True, key_type=None, stream=None):
    """Sorts every array of keys_list in place in one pass of the pipeline (tuned parameters are
    looked up for the mean array size and the first model's shape)."""
    cnt = len(keys_list)
    if cnt:
        eps, bucket_log2, polish_blocks = _tuned(
            models[0], sum(k.numel() for k in keys_list) // cnt, key_code(keys_list[0], key_type),
            precision, eps, bucket_log2, polish_blocks)
    kp = (C.c_void_p * cnt)(*[k.data_ptr() for k in keys_list])
    pp = None
    if payloads is not None:
        pp = (C.c_void_p * cnt)(*[0 if p is None else p.data_ptr() for p in payloads])
    ns = (C.c_uint64 * cnt)(*[k.numel() for k in keys_list])
    fs = (C.c_void_p * cnt)(*[mm.handle.value for mm in models])
    o = _sopts(m, eps, tau, precision, bucket_log2, None, None, not stats, False, polish_blocks)
    st = (L.Stats * cnt)() if stats else None
    L.check("nnsort_sort_batch", L.lib().nnsort_sort_batch(
        kp, pp, ns, cnt, key_code(keys_list[0], key_type), fs, C.byref(o), st, _stream(stream)))
    return [s.as_dict() for s in st] if stats else None


def workspace_bytes(n: int, dtype: int, with_payload: bool = False) -> int:
    return int(L.lib().nnsort_workspace_bytes(n, dtype, int(with_payload), None))


def mlp_pwl(params, layers, h1, h2=0):
    """Piecewise-linear form of the MLP (nnsort_mlp_pwl, host only): (breaks, slope, icept) float64
    arrays, segment i covering translated inputs [breaks[i], breaks[i+1]) with F = slope[i] x +
    icept[i] (breaks[0] = -inf)."""
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    cnt = C.c_uint32()
    lib = L.lib()
    lib.nnsort_mlp_pwl(layers, h1, h2, p.ctypes.data_as(C.c_void_p), None, None, None, 0, C.byref(cnt))
    n = cnt.value
    b, sl, ic = (np.empty(n, np.float64) for _ in range(3))
    L.check("nnsort_mlp_pwl", lib.nnsort_mlp_pwl(
        layers, h1, h2, p.ctypes.data_as(C.c_void_p), b.ctypes.data_as(C.c_void_p),
        sl.ctypes.data_as(C.c_void_p), ic.ctypes.data_as(C.c_void_p), n, C.byref(cnt)))
    return b, sl, ic


# ------------------------------------------------------------------- forward / backward
def mlp_forward(params, x, layers, h1, h2=0, stream=None):
    torch = _torch()
    y = torch.empty_like(x)
    L.check("nnsort_mlp_forward", L.lib().nnsort_mlp_forward(
        _ptr(params), layers, h1, h2, _ptr(x), x.numel(), _ptr(y), _stream(stream)))
    return y


def mlp_backward(params, x, gy, layers, h1, h2=0, want_gx=True, stream=None):
    torch = _torch()
    gp = torch.empty_like(params)
    gx = torch.empty_like(x) if want_gx else None
    L.check("nnsort_mlp_backward", L.lib().nnsort_mlp_backward(
        _ptr(params), layers, h1, h2, _ptr(x), _ptr(gy), x.numel(), _ptr(gp), _ptr(gx),
        _stream(stream)))
    return gp, gx


def mlp_loss_grad(params, x, label, layers, h1, h2=0, loss="mse", huber_delta=0.01, stream=None):
    torch = _torch()
    gp = torch.empty_like(params)
    lv = torch.empty(1, dtype=torch.float32, device=x.device)
    L.check("nnsort_mlp_loss_grad", L.lib().nnsort_mlp_loss_grad(
        _ptr(params), layers, h1, h2, _ptr(x), _ptr(label), x.numel(),
        {"mse": LOSS_MSE, "huber": LOSS_HUBER}.get(loss, loss), huber_delta, _ptr(lv), _ptr(gp),
        _stream(stream)))
    return lv, gp


def _make_autograd():
    torch = _torch()

    class NNSortMLPFunction(torch.autograd.Function):
        """y = f(x; params) with the library's forward kernel; backward through the library's
        hand-written backward kernel (fixed-order reductions)."""

        @staticmethod
        def forward(ctx, params, x, layers, h1, h2):
            ctx.save_for_backward(params, x)
            ctx.arch = (layers, h1, h2)
            return mlp_forward(params.contiguous(), x.contiguous(), layers, h1, h2)

        @staticmethod
        def backward(ctx, gy):
            params, x = ctx.saved_tensors
            layers, h1, h2 = ctx.arch
            gp, gx = mlp_backward(params.contiguous(), x.contiguous(), gy.contiguous(), layers, h1, h2,
                                  want_gx=ctx.needs_input_grad[1])
            return gp, gx, None, None, None

    return NNSortMLPFunction


class _LazyFn:
    _fn = None

    def __getattr__(self, name):
        if _LazyFn._fn is None:
            _LazyFn._fn = _make_autograd()
        return getattr(_LazyFn._fn, name)


NNSortMLPFunction = _LazyFn()


# ------------------------------------------------------------------------------- serving
class Server:
    """Continuous-batching sort server (nnsort_server_*): host arrays in, sorted in place."""

    def __init__(self, hbm_budget: int = 120 << 30, workers: int = 2, max_batch: int = 32,
                 max_batch_keys: int = 0, train: dict | None = None, sort: dict | None = None):
        SL = L.server_lib()
        o = L.ServerOpts()
        SL.nnsort_default_server_opts(C.byref(o))
        o.hbm_budget, o.workers, o.max_batch, o.max_batch_keys = hbm_budget, workers, max_batch, max_batch_keys
        o.train = _topts(**(train or {}))
        so = dict(m=1.25, eps=3, tau=1024, precision="fp32", bucket_log2=0)
        so.update(sort or {})
        o.sort = _sopts(so["m"], so["eps"], so["tau"], so["precision"], so["bucket_log2"], None, None,
                        False, False, so.get("polish_blocks", 0))
        self._h = C.c_void_p()
        L.check("nnsort_server_create", SL.nnsort_server_create(C.byref(o), C.byref(self._h)))
        self._keep = {}

    def submit(self, keys: np.ndarray, payload: np.ndarray | None = None, seed: int = 0) -> int:
        code = {np.dtype(np.float32): F32, np.dtype(np.float64): F64, np.dtype(np.uint32): U32,
                np.dtype(np.uint64): U64}[keys.dtype]
        assert keys.flags.c_contiguous and (payload is None or payload.flags.c_contiguous)
        t = C.c_uint64()
        L.check("nnsort_server_submit", L.lib().nnsort_server_submit(
            self._h, keys.ctypes.data_as(C.c_void_p),
            None if payload is None else payload.ctypes.data_as(C.c_void_p), keys.shape[0], code,
            seed, C.byref(t)))
        self._keep[t.value] = (keys, payload)
        return t.value

    def _result(self, fn, ticket):
        st = L.Stats()
        lat = C.c_double()
        rc = fn(self._h, ticket, C.byref(st), C.byref(lat))
        if rc == L.PENDING:
            return None
        self._keep.pop(ticket, None)
        L.check("nnsort_server_result", rc)
        return st.as_dict(), lat.value

    def poll(self, ticket: int):
        """(stats, latency_s) once finished, else None."""
        return self._result(L.lib().nnsort_server_poll, ticket)

    def wait(self, ticket: int):
        return self._result(L.lib().nnsort_server_wait, ticket)

    def close(self):
        if getattr(self, "_h", None):
            L.lib().nnsort_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        self.close()
