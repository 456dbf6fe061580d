"""The warm-start encoder's tensor-core convolutions (tcgen05 implicit GEMM,
BF16 operands, FP32 accumulation) against FP32 CPU convolutions of the same
BF16 values, and the encoder's training step against CPU autograd.

Tolerances: the GPU result is an FP32 sum of BF16 products, rounded to BF16
for BF16 outputs: |gpu - ref| <= 2^-8 |ref| + 1e-5 * sum|terms| (BF16
rounding of the output, FP32 summation in another order).  The encoder's
gradient is compared per weight tensor with the CPU network run on BF16
activations at the same points: 3e-2 of the tensor's largest entry (BF16
activations and gradients between the layers).
"""
import ctypes

import numpy as np
import pytest
import torch
import torch.nn.functional as F

from paper_2505_21319_gb300 import _binding as B
from paper_2505_21319_gb300 import api, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"
E = 32


def bf16(a):
    return torch.as_tensor(a, dtype=torch.float32).to(torch.bfloat16)


def rand_act(batch, C, seed, relu=False):
    g = torch.Generator().manual_seed(seed)
    x = torch.randn((batch, E, E, E, C), generator=g)
    return bf16(torch.relu(x) if relu else x)


def to_ncdhw(x):   # (n, x, y, z, c) -> (n, c, x, y, z)
    return x.float().permute(0, 4, 1, 2, 3).contiguous()


def w_to_torch(w, taps):   # (co, taps, ci) -> (co, ci, kx, ky, kz)
    co, _, ci = w.shape
    k = 3 if taps == 27 else 1
    return w.float().reshape(co, k, k, k, ci).permute(0, 4, 1, 2, 3).contiguous()


def conv_ref(x, w, taps):
    return F.conv3d(to_ncdhw(x), w_to_torch(w, taps), padding=1 if taps == 27 else 0).permute(0, 2, 3, 4, 1)


def err_flag():
    return torch.zeros(1, dtype=torch.int32, device=DEV)


def stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("cin,cout,taps,mode", [(64, 64, 27, 0), (64, 128, 27, 0), (64, 32, 27, 0), (128, 64, 27, 2),
                                                (128, 16, 1, 1), (64, 128, 1, 2), (128, 128, 27, 0)])
def test_conv_matches_cpu(cin, cout, taps, mode):
    batch = 2
    x = rand_act(batch, cin, seed=cin + cout + taps)
    g = torch.Generator().manual_seed(7)
    w = bf16(torch.randn((cout, taps, cin), generator=g) / np.sqrt(taps * cin))
    bias = torch.randn(cout, generator=g)
    ref = conv_ref(x, w, taps)                     # (n, x, y, z, cout) FP32
    terms = F.conv3d(to_ncdhw(x).abs(), w_to_torch(w, taps).abs(),
                     padding=1 if taps == 27 else 0).permute(0, 2, 3, 4, 1)
    mask = rand_act(batch, cout, seed=3) if mode == 2 else None
    if mode == 0:
        ref = torch.relu(ref + bias)
    elif mode == 1:
        ref = (ref + bias)[..., :13]
        terms = terms[..., :13]
    else:
        ref = torch.where(mask.float() > 0, ref, torch.zeros_like(ref))
    xd, wd = x.to(DEV), w.to(DEV)   # device copies held for the call
    bd = bias.to(DEV) if mode != 2 else None
    md = mask.to(DEV) if mask is not None else None
    out_ld = 13 if mode == 1 else cout
    out = torch.full((batch, E, E, E, out_ld), float("nan"), dtype=torch.float32 if mode == 1 else torch.bfloat16,
                     device=DEV)
    err = err_flag()
    B.check("efunc_conv3d_bf16", B.load().efunc_conv3d_bf16(
        xd.data_ptr(), batch, cin, wd.data_ptr(), cout, taps, bd.data_ptr() if bd is not None else None, mode,
        md.data_ptr() if md is not None else None, out.data_ptr(), out_ld, 13 if mode == 1 else cout,
        err.data_ptr(), stream()))
    torch.cuda.synchronize()
    assert err.item() == 0
    got = out.float().cpu()
    lim = (2.0 ** -8 if mode != 1 else 1e-6) * ref.abs() + 1e-5 * terms + 1e-6
    bad = (got - ref).abs() > lim
    assert not bad.any(), f"{bad.sum().item()} of {bad.numel()} outside; worst {((got - ref).abs() - lim).max():.3e}"


@pytest.mark.parametrize("dy_ld,cout,cin,taps", [(128, 128, 64, 27), (64, 64, 64, 27), (64, 16, 128, 1),
                                                 (128, 128, 128, 1)])
def test_wgrad_matches_cpu(dy_ld, cout, cin, taps):
    batch = 2
    dy = rand_act(batch, dy_ld, seed=dy_ld + cout)
    x = rand_act(batch, cin, seed=cin + 1, relu=True)
    k = 3 if taps == 27 else 1
    ref = torch.nn.grad.conv3d_weight(to_ncdhw(x), (dy_ld, cin, k, k, k), to_ncdhw(dy),
                                      padding=1 if taps == 27 else 0)   # (co, ci, kx, ky, kz)
    ref = ref.permute(0, 2, 3, 4, 1).reshape(dy_ld, taps, cin)[:cout]
    dw = torch.zeros((cout, taps, cin), device=DEV)
    err = err_flag()
    dyd, xd = dy.to(DEV), x.to(DEV)   # held: a temporary's memory could be handed to the next copy
    B.check("efunc_conv3d_wgrad_bf16", B.load().efunc_conv3d_wgrad_bf16(
        dyd.data_ptr(), dy_ld, cout, xd.data_ptr(), cin, batch, taps, dw.data_ptr(), err.data_ptr(), stream()))
    torch.cuda.synchronize()
    assert err.item() == 0
    got = dw.cpu()
    scale = ref.abs().max().item()
    assert (got - ref).abs().max().item() <= 1e-4 * scale, f"max err {(got - ref).abs().max().item():.3e} of {scale:.3e}"


class CpuEncoder(torch.nn.Module):
    """The encoder in FP32 on the CPU, with the BF16 rounding of the GPU path
    between the layers (activations and the weights' BF16 copies)."""

    def __init__(self, w):
        super().__init__()
        self.p = torch.nn.Parameter(w.clone())

    def split(self):
        p, o, out = self.p, 0, []
        for shape in ((32, 27), (32,), (64, 27, 32), (64,), (128, 27, 64), (128,), (13, 128), (13,)):
            n = int(np.prod(shape))
            out.append(p[o:o + n].reshape(shape))
            o += n
        return out

    def forward(self, sdf):
        w1, b1, w2, b2, w3, b3, w4, b4 = self.split()
        rb = lambda t: t + (t.to(torch.bfloat16).float() - t).detach()   # BF16 value, FP32 gradient
        x = sdf[:, None]
        a1 = rb(torch.relu(F.conv3d(x, w1.reshape(32, 3, 3, 3)[:, None], b1, padding=1)))
        a2 = rb(torch.relu(F.conv3d(a1, w_to_torch(rb(w2), 27), b2, padding=1)))
        a3 = rb(torch.relu(F.conv3d(a2, w_to_torch(rb(w3), 27), b3, padding=1)))
        out = F.conv3d(a3, rb(w4)[:, :, None, None, None], b4)
        return out.permute(0, 2, 3, 4, 1).reshape(sdf.shape[0], -1)


def _pairs(batch, seed):
    sdf = torch.stack([synth.sdf_grid_torch(synth.random_union(seed + i, n_prims=6), E, "cpu") for i in range(batch)])
    tgt = torch.stack([torch.from_numpy(synth.sdf_params(synth.random_union(seed + i, n_prims=6), E, seed=i)
                                        .reshape(-1)) for i in range(batch)])
    return sdf, tgt


def test_encoder_forward_and_gradient_match_cpu_autograd():
    batch = 2
    w = api.encoder_init(seed=1)
    sdf, tgt = _pairs(batch, 10)
    sw = torch.linspace(0.5, 2.0, 13)
    enc = api.Encoder(batch)
    wd = w.to(DEV)
    pred = enc.forward(wd, sdf.to(DEV)).cpu()
    grad, loss = enc.train_step(wd, sdf.to(DEV), tgt.to(DEV), sw.to(DEV))
    enc.status()
    cpu = CpuEncoder(w)
    pc = cpu(sdf)
    V = batch * E ** 3
    lc = ((pc.reshape(V, 13) - tgt.reshape(V, 13)) ** 2 * sw).sum() / V
    lc.backward()
    scale = pc.abs().max().item()
    assert (pred - pc.detach()).abs().max().item() <= 2e-2 * scale
    assert abs(loss.item() - lc.item()) <= 3e-2 * lc.item()
    g, gc = grad.cpu(), cpu.p.grad
    o = 0
    for name, n in (("W1", 864), ("b1", 32), ("W2", 55296), ("b2", 64), ("W3", 221184), ("b3", 128), ("W4", 1664),
                    ("b4", 13)):
        a, b = g[o:o + n], gc[o:o + n]
        assert (a - b).abs().max().item() <= 3e-2 * b.abs().max().item() + 1e-12, f"{name}"
        o += n


def test_encoder_training_lowers_the_loss():
    batch = 4
    w = api.encoder_init(seed=2).to(DEV)
    sdf, tgt = _pairs(batch, 20)
    sdf, tgt = sdf.to(DEV), tgt.to(DEV)
    enc = api.Encoder(batch)
    m, v = torch.zeros_like(w), torch.zeros_like(w)
    losses = []
    for step in range(1, 41):
        grad, loss = enc.train_step(w, sdf, tgt)
        losses.append(loss.item())
        api.efunc_adam_step(w, grad, m, v, step, lr=1e-3)
    enc.status()
    assert losses[-1] < 0.5 * losses[0]


def test_warm_start_pipeline_starts_closer_than_the_plain_initialisation():
    """The whole warm-start path on a few shapes: plain batched fits give the
    training pairs, the encoder trains on them, and its prediction for
    held-out shapes starts their fits at a lower held-out MAE than the
    N(0, 1e-3) initialisation (which predicts O ~ 0)."""
    from paper_2505_21319_gb300 import warmstart as W
    dev = torch.device(DEV)
    train = W.random_shapes(1000, 32)
    tp, _ = W.fit_plain(train, J=1 << 14, steps=200, seed=1, device=dev)
    w, losses, _ = W.train_encoder(W.sdf_grids(train, dev), tp, epochs=6, batch=8)
    assert losses[-1] < losses[0]
    ev = W.random_shapes(2000, 4)
    held = W.heldout_rows(ev, 1 << 13, seed=3, device=dev)
    pred, _ = W.predict(w, W.sdf_grids(ev, dev), batch=8)
    init = torch.cat([torch.from_numpy(synth.init_params(32, seed=i).reshape(1, -1)) for i in range(4)]).to(dev)
    st_w, mae_w, _ = W.fit_curves(ev, pred, J=1 << 14, max_steps=50, every=25, seed=4, held=held)
    st_p, mae_p, _ = W.fit_curves(ev, init, J=1 << 14, max_steps=50, every=25, seed=4, held=held)
    assert np.median(mae_w[0]) < np.median(mae_p[0])
    assert np.isfinite(mae_w).all() and np.isfinite(mae_p).all()
