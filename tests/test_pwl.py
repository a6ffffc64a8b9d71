"""The compiled piecewise-linear form of f (nnsort_mlp_pwl, host code, no GPU): equal to the oracle's
binary64 forward pass everywhere (random points and both sides of every break), continuous at the
breaks, within the segment-count bound, and the closed form of a one-unit network."""
import numpy as np
import pytest

from oracle import oracle as orc
import workloads as W

nns = pytest.importorskip("paper_1907_08817_gb300")


def _eval(brk, sl, ic, x):
    i = np.searchsorted(brk, x, side="right") - 1
    return sl[i] * x + ic[i]


def _check(params, layers, h1, h2, xs):
    brk, sl, ic = nns.mlp_pwl(params, layers, h1, h2)
    assert brk[0] == -np.inf and np.all(np.diff(brk[1:]) > 0)
    bound = h1 + 1 if layers == 1 else 1 + h1 + (h1 + 1) * h2
    assert 1 <= brk.shape[0] <= bound
    y64 = orc.mlp_forward_f64(layers, h1, h2, params, xs)
    yp = _eval(brk, sl, ic, xs)
    scale = 1.0 + np.abs(y64)
    np.testing.assert_array_less(np.abs(yp - y64) / scale, 1e-9)
    # both sides of every break, and continuity across it
    b = brk[1:]
    eps = 1e-7 * (1.0 + np.abs(b))
    for side in (b - eps, b + eps):
        np.testing.assert_array_less(np.abs(_eval(brk, sl, ic, side) - orc.mlp_forward_f64(layers, h1, h2, params, side))
                                     / (1.0 + np.abs(side)), 1e-6)
    left = sl[:-1] * b + ic[:-1]
    right = sl[1:] * b + ic[1:]
    np.testing.assert_array_less(np.abs(left - right) / (1.0 + np.abs(left)), 1e-9)
    return brk


@pytest.mark.parametrize("layers,h", [(1, 8), (1, 32), (2, 16), (2, 64)])
def test_pwl_matches_binary64_forward_random_init(layers, h):
    h2 = h if layers == 2 else 0
    rs = np.random.RandomState(h + layers)
    xs = np.concatenate([rs.uniform(-0.5, 1.5, 20000), rs.uniform(-50, 50, 2000)])
    for seed in range(3):
        _check(orc.init_params(layers, h, h2, seed), layers, h, h2, xs)


@pytest.mark.parametrize("layers,h", [(1, 32), (2, 32)])
def test_pwl_matches_binary64_forward_trained(layers, h):
    keys = W.lognormal_dup_f32(50_000, 7, sigma=2.0)
    h2 = h if layers == 2 else 0
    om, _, _ = orc.train(keys, layers, h, h2, orc.ORDBITS, sample_n=2000, steps=60, lr=1e-2, seed=3)
    xs = orc.translate_f64(keys, om.norm)
    brk = _check(om.params, layers, h, h2, xs)
    assert brk.shape[0] > 2


def test_pwl_closed_form_one_unit():
    # F(x) = relu(x): two segments, 0 below 0 and x above
    p = np.zeros(3 * 2 + 1, np.float32)
    p[0], p[2], p[4] = 1.0, 0.0, 1.0  # W1 = [1, 0], b1 = [0, 0], W3 = [1, 0], b3 = 0
    brk, sl, ic = nns.mlp_pwl(p, 1, 2, 0)
    np.testing.assert_array_equal(brk, [-np.inf, 0.0])
    np.testing.assert_array_equal(sl, [0.0, 1.0])
    np.testing.assert_array_equal(ic, [0.0, 0.0])
