"""GPU parity of the learned tracking warm-start network against the FP64
oracle (oracle/cnn.py).

The GPU multiplies BF16 operands (weights, stored activations, stored
upstream gradients) and accumulates in FP32; the oracle runs in FP64 on the
BF16-rounded weights and input.  Bars, in relative L2 norm per tensor:
forward output <= 1e-2, each parameter gradient <= 2e-2.

A ReLU mask is a discontinuity: where a pre-activation lies within the
forward's rounding difference of zero (about 1e-3 of its scale here), the GPU
and the oracle may disagree on the mask, and that element's gradient then
differs by its full size (one flip among the 256 hidden units moves the
dense-1 gradient by several per cent).  The gradient parity cases therefore
use networks whose every pre-activation has a margin from zero by
construction: inputs >= 0, and in every ReLU layer each output channel either
has weights >= 0 and bias +0.1 (always active) or weights <= 0 and bias -0.1
(always inactive).  Every GEMM, im2col / col2im, bias and mask path still
runs.  With random weights of both signs the forward output and the output
layer's gradients (downstream of every mask) are compared.
"""
import numpy as np
import pytest
import torch

from oracle import cnn as C

pytestmark = pytest.mark.gpu


def bf16_round(a):
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def rel_l2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def random_params(seed):
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in C.param_shapes():
        if name.endswith(".b"):
            p[name] = rng.normal(0, 0.05, shp).astype(np.float32)
        else:
            fan_in = int(np.prod(shp[1:]))
            p[name] = rng.normal(0, np.sqrt(2.0 / fan_in), shp).astype(np.float32)
    return p


@pytest.fixture(scope="module")
def ws():
    from paper_2312_10070_gb300 import warmstart as W
    return W


def signed_params(seed, frac_active=0.75):
    """Parameters with a sign per ReLU output channel (see the module doc)."""
    rng = np.random.default_rng(seed)
    p = {}
    shapes = dict(C.param_shapes())
    relu_layers = [f"conv{i}" for i in range(len(C.CONV))] + ["fc0"]
    for name in relu_layers:
        w = np.abs(rng.normal(0, 1, shapes[name + ".w"]))
        co = w.shape[0]
        sign = np.where(rng.random(co) < frac_active, 1.0, -1.0)
        fan_in = int(np.prod(w.shape[1:]))
        w = sign.reshape((co,) + (1,) * (w.ndim - 1)) * w / (0.5 * fan_in)
        p[name + ".w"] = w.astype(np.float32)
        p[name + ".b"] = (0.1 * sign).astype(np.float32)
    p["fc1.w"] = rng.normal(0, np.sqrt(1.0 / 256), shapes["fc1.w"]).astype(np.float32)
    p["fc1.b"] = rng.normal(0, 0.05, shapes["fc1.b"]).astype(np.float32)
    return p


def run_gpu(ws, p32, x, d_out):
    net = ws.WarmStartNet(max_batch=8, seed=0)
    flat = C.flatten({k: v.astype(np.float64) for k, v in p32.items()}).astype(np.float32)
    net.set_params(torch.from_numpy(flat).cuda())
    np.testing.assert_array_equal(net.get_params().cpu().numpy(), flat)
    out = net.forward(torch.from_numpy(x).cuda())
    g = net.backward(torch.from_numpy(d_out).cuda())
    torch.cuda.synchronize()
    return out.cpu().numpy(), C.unflatten(g.cpu().numpy())


def oracle_bf16(p32):
    return {k: (v.astype(np.float64) if k.endswith(".b") else bf16_round(v)) for k, v in p32.items()}


@pytest.mark.parametrize("batch", [1, 3, 8])
def test_forward_backward_match_oracle(ws, batch):
    rng = np.random.default_rng(10 + batch)
    p32 = signed_params(20 + batch)
    x = rng.random((batch, C.IN_H, C.IN_W, C.IN_C)).astype(np.float32)
    d_out = rng.standard_normal((batch, 6)).astype(np.float32)
    out, got = run_gpu(ws, p32, x, d_out)
    pr = oracle_bf16(p32)
    ref_out, cache = C.forward(pr, bf16_round(x))
    # the construction's margin: every pre-activation at least 0.05 from zero
    for _, _, z in cache[0]:
        assert np.abs(z).min() > 0.05
    assert np.abs(cache[2]).min() > 0.05
    ref_g = C.backward(pr, cache, d_out.astype(np.float64))
    assert rel_l2(out, ref_out) <= 1e-2
    errs = {name: rel_l2(got[name], ref_g[name]) for name, _ in C.param_shapes()}
    bad = {k: e for k, e in errs.items() if not e <= 2e-2}
    assert not bad, (bad, errs)


def test_random_weights_forward(ws):
    """Random signed weights: the forward output, and the output layer's
    gradients (no ReLU mask after them), against the storage-rounded and the
    plain oracle."""
    p32 = random_params(30)
    pr = oracle_bf16(p32)
    rng = np.random.default_rng(1000)
    x = rng.standard_normal((2, C.IN_H, C.IN_W, C.IN_C)).astype(np.float32)
    d_out = rng.standard_normal((2, 6)).astype(np.float32)
    out, got = run_gpu(ws, p32, x, d_out)
    ref_out, cache = C.forward(pr, bf16_round(x), rnd=bf16_round)
    ref_g = C.backward(pr, cache, d_out.astype(np.float64), rnd=bf16_round)
    plain_out, _ = C.forward(pr, bf16_round(x))
    assert rel_l2(out, ref_out) <= 1e-2 and rel_l2(out, plain_out) <= 1e-2
    for name in ("fc1.w", "fc1.b"):
        assert rel_l2(got[name], ref_g[name]) <= 2e-2, name


def test_train_step_loss_and_first_adam_step(ws):
    """The loss equals the oracle's weighted MSE of the forward output, and
    the first Adam step moves each parameter by lr * g / (|g| + eps) with g the
    gradient backward returns for d_out = dL/dout."""
    rng = np.random.default_rng(7)
    B = 4
    x = torch.from_numpy(rng.standard_normal((B, C.IN_H, C.IN_W, C.IN_C)).astype(np.float32)).cuda()
    tgt = torch.from_numpy(rng.standard_normal((B, 6)).astype(np.float32) * 0.05).cuda()
    w = (1.0, 2.0, 1.0, 0.5, 1.0, 3.0)
    net = ws.WarmStartNet(max_batch=B, seed=3)
    p0 = net.get_params()
    out = net.forward(x)
    L_ref, d_ref = C.loss(out.cpu().numpy(), tgt.cpu().numpy(), w)
    g = net.backward(torch.from_numpy(d_ref.astype(np.float32)).cuda())
    cfg = ws.WarmstartConfig(lr=1e-3, eps=1e-8, weights=w)
    loss = net.train_step(x, tgt, cfg)
    p1 = net.get_params()
    torch.cuda.synchronize()
    assert abs(loss.item() - L_ref) <= 1e-5 * max(1.0, abs(L_ref))
    step = (p0 - p1).double().cpu().numpy()
    gd = g.double().cpu().numpy()
    pred = 1e-3 * gd / (np.abs(gd) + 1e-8)
    big = np.abs(gd) > 1e-4 * np.abs(gd).max()
    np.testing.assert_allclose(step[big], pred[big], rtol=1e-3, atol=1e-7)


def test_training_fits_a_fixed_batch(ws):
    rng = np.random.default_rng(8)
    B = 16
    x = torch.from_numpy(rng.standard_normal((B, C.IN_H, C.IN_W, C.IN_C)).astype(np.float32)).cuda()
    tgt = torch.from_numpy(rng.uniform(-0.05, 0.05, (B, 6)).astype(np.float32)).cuda()
    net = ws.WarmStartNet(max_batch=B, seed=4)
    cfg = ws.WarmstartConfig(lr=1e-3)
    first = net.train_step(x, tgt, cfg).item()
    for _ in range(200):
        last = net.train_step(x, tgt, cfg)
    assert last.item() < 0.05 * first


def test_make_input_matches_oracle(ws):
    rng = np.random.default_rng(9)
    h, w = 680, 1200
    rgb_r = rng.random((3, 120, 160)).astype(np.float32)
    d_r = rng.uniform(0.5, 4, (120, 160)).astype(np.float32)
    d_r[rng.random((120, 160)) < 0.1] = 0
    rgb_i = rng.random((3, h, w)).astype(np.float32)
    d_i = rng.uniform(0.5, 4, (h, w)).astype(np.float32)
    d_i[rng.random((h, w)) < 0.2] = 0
    d_i[0:20, 0:20] = 0  # a whole box without valid depth
    T = lambda a: torch.from_numpy(a).cuda()
    got = ws.make_input(T(rgb_r), T(d_r), T(rgb_i), T(d_i), 5.0).cpu().numpy()
    r_i, dd_i = C.box_downsample(rgb_i, d_i, 120, 160)
    ref = C.residual_input(rgb_r, d_r, r_i, dd_i, 5.0)
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-6)


def test_invalid_calls(ws):
    from paper_2312_10070_gb300 import _lib as L
    net = ws.WarmStartNet(max_batch=2, seed=0)
    x = torch.zeros(3, C.IN_H, C.IN_W, C.IN_C, device="cuda")
    with pytest.raises(L.GsrError):
        net.forward(x)  # batch above max_batch
    with pytest.raises(L.GsrError):
        net.backward(torch.zeros(2, 6, device="cuda"))  # no forward of that batch yet


@pytest.mark.parametrize("batch", [1, 5])
def test_tcgen05_forward_matches_mma_sync(ws, batch):
    """The tcgen05 forward products agree with the mma.sync ones (same BF16
    operands, FP32 accumulation in a different order) on every layer."""
    rng = np.random.default_rng(40 + batch)
    p32 = signed_params(50 + batch)
    x = torch.from_numpy(rng.random((batch, C.IN_H, C.IN_W, C.IN_C)).astype(np.float32)).cuda()
    net = ws.WarmStartNet(max_batch=8, seed=0)
    flat = C.flatten({k: v.astype(np.float64) for k, v in p32.items()}).astype(np.float32)
    net.set_params(torch.from_numpy(flat).cuda())
    net.set_kernels(0)      # every forward product on tcgen05
    out_tc = net.forward(x).cpu().numpy()
    net.check_status()
    net.set_kernels(-1)     # none
    out_ms = net.forward(x).cpu().numpy()
    assert rel_l2(out_tc, out_ms) <= 2e-3, (out_tc, out_ms)
