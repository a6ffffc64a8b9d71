"""GPU training path (Sec. "Training"): sample + labels, forward, hand-written backward, Adam,
against the CPU oracle (binary64 analytic gradients, binary64 training)."""
import numpy as np
import pytest

from helpers import lib_model, oracle_model, stats_core, to_dev
from oracle import oracle as orc
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)
import paper_1907_08817_gb300 as nns  # noqa: E402


@pytest.mark.parametrize("dtype", ["f32", "u64", "f64"])
@pytest.mark.parametrize("translate", [orc.ORDBITS, orc.VALUE])
def test_sample_labels_bit_exact(dtype, translate):
    if dtype == "f32":
        keys = W.lognormal_dup_f32(300_000, 2, sigma=2.0)
    elif dtype == "u64":
        keys, _ = W.gauss_mix_u64(300_000, 3)
    else:
        keys = W.normal_f32(300_000, 4).astype(np.float64)
    dk, kt = to_dev(keys)
    for S in (1, 1000, 65_537):
        x, lab, rows, norm = nns.sample_labels(dk, S, seed=5, translate=translate, key_type=kt)
        orows, onm, ox, olab = orc.sample_labels(keys, S, 5, translate)
        np.testing.assert_array_equal(rows.cpu().numpy().astype(np.uint32), orows.astype(np.uint32))
        np.testing.assert_array_equal(x.cpu().numpy().view(np.uint32), ox.view(np.uint32))
        np.testing.assert_array_equal(lab.cpu().numpy().view(np.uint32), olab.view(np.uint32))
        assert norm["lo_bits"] == onm.lo_bits and norm["scale"] == onm.scale


@pytest.mark.parametrize("arch", [(1, 32, 0), (2, 16, 16), (2, 64, 64), (2, 2, 6), (1, 5, 0)])
def test_forward_bit_exact(arch):
    layers, h1, h2 = arch
    p = orc.init_params(layers, h1, h2, 3)
    x = np.concatenate([W.uniform_f32(10_000, 1), np.array([-0.5, 0.0, 1.0, 1.5], np.float32)])
    y = nns.mlp_forward(torch.from_numpy(p).cuda(), torch.from_numpy(x).cuda(), layers, h1, h2)
    oy = orc.mlp_forward_f32(layers, h1, h2, p, x)
    np.testing.assert_array_equal(y.cpu().numpy().view(np.uint32), oy.view(np.uint32))


@pytest.mark.parametrize("arch", [(1, 32, 0), (2, 16, 16), (2, 64, 64), (2, 2, 6)])
@pytest.mark.parametrize("loss", ["mse", "huber"])
def test_loss_gradient_against_binary64(arch, loss):
    layers, h1, h2 = arch
    rs = np.random.RandomState(7)
    p = orc.init_params(layers, h1, h2, 11)
    n = 50_000
    x = rs.uniform(0, 1, n).astype(np.float32)
    lab = np.sort(rs.uniform(0, 1, n)).astype(np.float32)
    lv, g = nns.mlp_loss_grad(torch.from_numpy(p).cuda(), torch.from_numpy(x).cuda(),
                              torch.from_numpy(lab).cuda(), layers, h1, h2, loss=loss,
                              huber_delta=0.05)
    code = orc.HUBER if loss == "huber" else orc.MSE
    oL, og, _ = orc.mlp_loss_grad_f64(layers, h1, h2, p.astype(np.float64), x.astype(np.float64),
                                      lab.astype(np.float64), code, 0.05)
    gg = g.cpu().numpy().astype(np.float64)
    scale = np.abs(og).max()
    assert np.max(np.abs(gg - og)) <= 1e-4 * scale + 1e-7
    assert abs(float(lv.item()) - oL) <= 1e-4 * abs(oL) + 1e-7


def test_autograd_function_and_input_gradient():
    layers, h1, h2 = 2, 16, 16
    rs = np.random.RandomState(9)
    p = orc.init_params(layers, h1, h2, 2)
    n = 4096
    x = rs.uniform(0, 1, n).astype(np.float32)
    w = rs.uniform(-1, 1, n).astype(np.float32)
    pt = torch.from_numpy(p).cuda().requires_grad_(True)
    xt = torch.from_numpy(x).cuda().requires_grad_(True)
    y = nns.NNSortMLPFunction.apply(pt, xt, layers, h1, h2)
    (y * torch.from_numpy(w).cuda()).sum().backward()
    # s = sum_i w_i y_i equals n * mean loss of a linear "loss" -> compare with binary64 via the
    # MSE form: d/dp sum_i w_i y_i = sum_i w_i dy_i/dp. Build it from the oracle by choosing labels
    # label_i = y_i - w_i * n / 2, for which MSE's gradient weight 2 r_i / n equals w_i.
    y64 = orc.mlp_forward_f64(layers, h1, h2, p.astype(np.float64), x.astype(np.float64))
    lab = y64 - w.astype(np.float64) * n / 2.0
    _, og, ogx = orc.mlp_loss_grad_f64(layers, h1, h2, p.astype(np.float64), x.astype(np.float64),
                                       lab, orc.MSE)
    g = pt.grad.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(g - og)) <= 1e-4 * np.abs(og).max() + 1e-6
    gx = xt.grad.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(gx, ogx * 1.0, rtol=1e-3, atol=1e-4 * np.abs(ogx).max())
    # reproducible: fixed-order reductions give identical gradients run to run
    pt2 = pt.detach().clone().requires_grad_(True)
    y2 = nns.NNSortMLPFunction.apply(pt2, xt.detach(), layers, h1, h2)
    (y2 * torch.from_numpy(w).cuda()).sum().backward()
    assert torch.equal(pt2.grad, pt.grad)


@pytest.mark.parametrize("cfg", [
    dict(layers=1, h1=32, h2=0, translate=orc.VALUE, sample_n=10_000, steps=100, batch=0),
    dict(layers=2, h1=16, h2=16, translate=orc.ORDBITS, sample_n=20_000, steps=100, batch=0),
    dict(layers=1, h1=16, h2=0, translate=orc.ORDBITS, sample_n=20_000, steps=60, batch=512),
])
def test_device_training_tracks_binary64_training(cfg):
    keys = W.lognormal_dup_f32(1_000_000, 2, sigma=2.0) if cfg["translate"] == orc.ORDBITS \
        else W.uniform_f32(1_000_000, 0)
    dk, kt = to_dev(keys)
    model, hist = nns.train(dk, seed=0, lr=1e-2, **cfg)
    om, p64, ohist = orc.train(keys, seed=0, lr=1e-2, **cfg)
    _, p = model.describe()
    # same data, same initialisation, same batches: the trajectories agree to binary32 noise
    assert abs(hist[0] - ohist[0]) <= 1e-5 * abs(ohist[0]) + 1e-7
    np.testing.assert_allclose(hist, ohist, rtol=2e-3, atol=1e-6)
    assert np.max(np.abs(p - p64)) <= 2e-3 * np.abs(p64).max()
    assert hist[-1] < hist[0]


@pytest.mark.parametrize("arch", [(1, 16, 0), (2, 32, 32), (2, 64, 64)])
def test_monotone_training_on_device(arch):
    """Sign-structured training: the device run follows the oracle's projected binary64 run, and
    the resulting positions never decrease with the key, in binary32 and BF16 arithmetic, so the
    polish finds no out-of-order element and no bucket seam needs repair."""
    layers, h1, h2 = arch
    keys = W.lognormal_dup_f32(2_000_000, 12, sigma=2.0)
    dk, _ = to_dev(keys)
    cfg = dict(layers=layers, h1=h1, h2=h2, translate=orc.ORDBITS, sample_n=20_000, steps=100,
               batch=4096, seed=4)
    model, hist = nns.train(dk, lr=1e-2, monotone=True, **cfg)
    om, p64, ohist = orc.train(keys, lr=1e-2, monotone=True, **cfg)
    np.testing.assert_allclose(hist, ohist, rtol=5e-3, atol=1e-6)
    _, p = model.describe()
    assert np.max(np.abs(p - p64)) <= 5e-3 * np.abs(p64).max()
    precs = ["fp32"] + (["bf16"] if layers == 2 else [])
    for prec in precs:
        k = dk.clone()
        slots, _ = nns.predict(k, model, precision=prec, want_y=False)
        order = torch.argsort(k, stable=True)
        s_sorted = slots[order]
        assert bool((s_sorted[1:] >= s_sorted[:-1]).all())
        st = nns.sort(k, None, model, precision=prec)
        assert sum(st["out_of_order"]) == 0 and st["repaired"] == 0
        assert torch.equal(k, torch.sort(dk).values)


def test_trained_model_gains_over_untrained_and_linear():
    """What the learned network buys: fewer conflicts and a smaller traditional-sort share than the
    same pipeline with the untrained network or with the plain min-max (linear) map."""
    keys = W.lognormal_dup_f32(2_000_000, 2, sigma=2.0)
    dk, _ = to_dev(keys)
    trained, _ = nns.train(dk, layers=1, h1=32, translate="value", sample_n=20_000, steps=300, seed=0)
    d, _ = trained.describe()
    untrained = nns.Model.create(orc.F32, 1, 32, 0, orc.init_params(1, 32, 0, 0), orc.VALUE,
                                 d["lo_bits"], d["lo_val"], d["scale"])
    linear = nns.Model.create(orc.F32, 1, 1, 0, np.array([1.0, 0.0, 1.0, 0.0], np.float32),
                              orc.VALUE, d["lo_bits"], d["lo_val"], d["scale"])
    res = {}
    for name, f in (("trained", trained), ("untrained", untrained), ("linear", linear)):
        k = dk.clone()
        res[name] = nns.sort(k, None, f, eps=3, tau=0)
        assert torch.equal(k, torch.sort(dk).values)
    assert res["trained"]["sigma"][0] < res["linear"]["sigma"][0]
    assert res["trained"]["sigma"][0] < res["untrained"]["sigma"][0]
    assert res["trained"]["trad_rate"] < res["linear"]["trad_rate"]


def test_batched_training_tracks_binary64_training():
    """nnsort_train_batch (one block per model: sample, sort, labels, every Adam step on chip):
    model j uses seed seed + j and its own sample size; its normaliser equals the oracle's from the
    same sample bit for bit, and its loss history and weights follow the oracle's binary64 training
    of that array to binary32 noise, for float32, float64 and uint64 keys, full batch and
    minibatch, hidden widths 8, 16 and 32."""
    arrs = [a for _, a in W.batch_arrays(5, seed=9, lo=2000, hi=400_000)]
    arrs.append(W.lognormal_dup_f32(1_700_000, 4, sigma=2.0))   # a 16,384-key sample (the limit)
    arrs.append(W.uniform_f32(900, 3))                          # a 9-key sample
    cases = [(arrs, [max(9, a.shape[0] // 100) for a in arrs[:-2]] + [16384, 9], 16, 0),
             ([rs_normal(300_000, 5)], [3000], 8, 64),
             ([W.gauss_mix_u64(500_000, 3)[0]], [5000], 32, 0)]
    for arrays, S, h, batch in cases:
        dks = [to_dev(a)[0] for a in arrays]
        kt = to_dev(arrays[0])[1]
        models, hist = nns.train_batch(dks, sample_ns=S, key_type=kt, layers=1, h1=h, steps=100,
                                       batch=batch, lr=1e-2, seed=5)
        for j, (a, m, s_j) in enumerate(zip(arrays, models, S)):
            om, p64, ohist = orc.train(a, 1, h, 0, orc.ORDBITS, sample_n=s_j, steps=100,
                                       batch=batch, lr=1e-2, seed=5 + j)
            d, p = m.describe()
            assert (d["lo_bits"], d["lo_val"], d["scale"]) == (om.norm.lo_bits, om.norm.lo_val,
                                                              om.norm.scale)
            assert abs(hist[j][0] - ohist[0]) <= 1e-5 * abs(ohist[0]) + 1e-7
            np.testing.assert_allclose(hist[j], ohist, rtol=2e-3, atol=1e-6)
            assert np.max(np.abs(p - p64)) <= 2e-3 * np.abs(p64).max()
    # two hidden layers are trained by nnsort_train, not in a batch
    with pytest.raises(nns.NNSortError) as ei:
        nns.train_batch([to_dev(arrs[0])[0]], layers=2, h1=16, h2=16, sample_n=100)
    assert ei.value.status == -7


def rs_normal(n, seed):
    return np.random.RandomState(seed).standard_normal(n)
