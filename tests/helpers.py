"""Shared test helpers: moving numpy arrays to the device and building the oracle's model from the
library's model description (parameters are copied, never recomputed)."""
import numpy as np

from oracle import oracle as orc


def to_dev(a: np.ndarray):
    """(device tensor, key_type) for a numpy key array; unsigned keys travel as same-width ints."""
    import torch
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        return torch.from_numpy(a.view(np.int64)).cuda(), "u64"
    if a.dtype == np.uint32:
        return torch.from_numpy(a.view(np.int32)).cuda(), "u32"
    return torch.from_numpy(a).cuda(), None


def from_dev(t, like: np.ndarray) -> np.ndarray:
    return t.cpu().numpy().view(like.dtype)


def oracle_model(model) -> orc.Model:
    d, p = model.describe()
    nm = orc.Norm(d["dtype"], d["translate"], d["lo_bits"], d["lo_val"], d["scale"],
                  np.float32(d["lo_val"]), np.float32(d["scale"]))
    return orc.Model(d["layers"], d["h1"], d["h2"], nm, p)


def lib_model(om: orc.Model):
    import paper_1907_08817_gb300 as nns
    nm = om.norm
    return nns.Model.create(nm.dtype, om.layers, om.h1, om.h2, om.params, nm.translate, nm.lo_bits,
                            nm.lo_val, nm.scale)


def bits(a: np.ndarray) -> np.ndarray:
    """Exact bit patterns for bit-for-bit comparison of keys."""
    return a.view({4: np.uint32, 8: np.uint64}[a.dtype.itemsize])


def stats_core(st: dict) -> dict:
    return {k: st[k] for k in ("t", "w_size", "placed", "out_of_order")}
