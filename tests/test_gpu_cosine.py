"""GPU parity of the cosine-series decomposition (Sec. 4.4) through the C
ABI against the FP64 oracle.

Tolerances (FP32 kernel vs FP64 oracle), per query:
  S               |gpu - ref| <= sum_b |w_b| tol(O_b) + (B + 8) u sum_b |w_b O_b|
                  tol(O_b) = max(1e-6 + 1e-5 |O_b|, 4 u kappa_b), the default
                  model's forward tolerance for each band (kappa_b from the
                  oracle); the second term covers the band weights (three FP32
                  cos(b pi x) factors of about one ulp each, from an exact split
                  of b x, and two products: 6u) and the B-term sum
  dL/dparams      per band and channel group (b, o, d): max |gpu - ref| <=
                  1e-4 max |ref| of the group
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2505_21319_gb300 import api, synth
from test_gpu_parity import lb32, mixed_queries, to_dev

pytestmark = pytest.mark.gpu

DEV = "cuda"
U32 = 2.0 ** -24


def band_params(R, B, seed, shaped=True):
    """B bands of Config-G-6 parameters (B, R^3, 5); band 0 shaped like a
    fitted grid of a random union, the others small corrections."""
    out = np.empty((B, R ** 3, 5), np.float32)
    shape = synth.random_union(seed) if shaped else None
    for b in range(B):
        p = synth.variant_params(shape if b == 0 else None, R, 1, 1, 1, seed=seed + b)
        if b > 0 and shaped:
            p[:, 1:] *= 0.1
        out[b] = p
    return out


def S_tolerance(p, q, R, B, lb):
    b = np.arange(B)[None, :]
    w = np.cos(b * np.pi * q[:, 0:1]) * np.cos(b * np.pi * q[:, 1:2]) * np.cos(b * np.pi * q[:, 2:3])
    tol = np.zeros(q.shape[0])
    mag = np.zeros(q.shape[0])
    for k in range(B):
        O, _, kap, _ = oracle.variant_forward(p[k], q, R, 1, 1, 1, log_beta0=lb, want_diag=True)
        tol += np.abs(w[:, k]) * np.maximum(1e-6 + 1e-5 * np.abs(O), 4 * U32 * kap)
        mag += np.abs(w[:, k] * O)
    return tol + (B + 8) * U32 * mag


def assert_cosine_grad_close(gpu, ref, what, rtol=1e-4, b_floor=None):
    """b_floor: per band, an absolute bound added for the log-scale group
    (when its exact gradient vanishes and the kernel's value is rounding)."""
    gpu = np.asarray(gpu, dtype=np.float64).reshape(ref.shape)
    for b in range(ref.shape[0]):
        for name, cols in (("b", [0]), ("o", [1]), ("d", [2, 3, 4])):
            scale = np.abs(ref[b][:, cols]).max()
            err = np.abs(gpu[b][:, cols] - ref[b][:, cols]).max()
            floor = b_floor[b] if (b_floor is not None and name == "b") else 0.0
            assert err <= rtol * scale + floor + 1e-30, f"{what} band {b} {name}: max err {err:.3e} vs {scale:.3e}"


@pytest.mark.parametrize("R,B,J", [(4, 1, 2001), (4, 5, 3001), (16, 2, 30011), (16, 8, 20000), (8, 16, 5000)])
def test_cosine_forward_matches_oracle(R, B, J):
    p = band_params(R, B, seed=R + B)
    qo = mixed_queries(R, J, seed=R * B)
    lb = lb32(R)
    S = api.efunc_cosine_forward(B, to_dev(p).reshape(-1), to_dev(qo), log_beta0=lb).cpu().numpy()
    ref = oracle.cosine_forward(p, qo[:, :3], R, B, log_beta0=lb)
    lim = S_tolerance(p, qo[:, :3].astype(np.float64), R, B, lb)
    err = np.abs(S.astype(np.float64) - ref)
    bad = np.flatnonzero(~(err <= lim))
    assert bad.size == 0, f"R={R} B={B}: {bad.size} of {J}; idx {bad[:5]} gpu {S[bad[:5]]} ref {ref[bad[:5]]}"


@pytest.mark.parametrize("R,B,J", [(5, 1, 3001), (8, 3, 20000), (16, 8, 40000)])
def test_cosine_backward_matches_oracle(R, B, J):
    p = band_params(R, B, seed=3 * R + B)
    qo = mixed_queries(R, J, seed=R + 7 * B)
    gS = (synth.rng(B).standard_normal(J) / J).astype(np.float32)
    grad = api.efunc_cosine_backward(B, to_dev(p).reshape(-1), to_dev(qo), to_dev(gS), log_beta0=lb32(R))
    g_ref = oracle.cosine_backward(p, qo[:, :3], gS, R, B, log_beta0=lb32(R))
    assert_cosine_grad_close(grad.cpu().numpy(), g_ref, f"R={R} B={B}")


def test_cosine_one_band_agrees_with_config_g6():
    """B = 1 is Config-G-6: the cosine kernels and the variant kernels agree
    within their oracle tolerance."""
    R, J = 16, 30000
    p = band_params(R, 1, seed=4)
    qo = mixed_queries(R, J, seed=9)
    lb = lb32(R)
    S = api.efunc_cosine_forward(1, to_dev(p).reshape(-1), to_dev(qo), log_beta0=lb).cpu().numpy()
    O = api.efunc_variant_forward("G-6", to_dev(p[0]).reshape(-1), to_dev(qo), log_beta0=lb).cpu().numpy()
    lim = S_tolerance(p, qo[:, :3].astype(np.float64), R, 1, lb)
    assert np.all(np.abs(S - O) <= 2 * lim)


@pytest.mark.parametrize("loss", ["l1", "mse"])
def test_cosine_fit_step_gradient_and_loss(loss):
    """One fused step with lr = 0 exposes the gradient of the loss on S
    through Adam's first moment; stats hold loss and MAE.  L1 targets sit at
    least 1e-3 from the oracle's S."""
    R, B, J = 16, 4, 50000
    p = band_params(R, B, seed=21)
    qo = mixed_queries(R, J, seed=22)
    lb = lb32(R)
    S_ref = oracle.cosine_forward(p, qo[:, :3], R, B, log_beta0=lb)
    g = synth.rng(23)
    qo[:, 3] = (S_ref + g.uniform(1e-3, 0.1, J) * np.where(g.integers(0, 2, J) == 0, -1.0, 1.0)).astype(np.float32)
    n = p.size
    pd, m, v = to_dev(p).reshape(-1), torch.zeros(n, device=DEV), torch.zeros(n, device=DEV)
    stats = torch.zeros(2, device=DEV)
    api.efunc_cosine_fit(B, pd, m, v, to_dev(qo), steps=1, loss=loss, stats=stats, lr=0.0, log_beta0=lb)
    gS, L, mae = oracle.loss_grad(S_ref, qo[:, 3].astype(np.float64), oracle.L1 if loss == "l1" else oracle.MSE)
    g_ref = oracle.cosine_backward(p, qo[:, :3], gS, R, B, log_beta0=lb)
    assert_cosine_grad_close(m.cpu().numpy() / 0.1, g_ref, f"fit {loss}")
    s = stats.cpu().numpy()
    assert abs(s[0] - L) <= 1e-5 * abs(L) + 1e-7
    assert abs(s[1] - mae) <= 1e-5 * abs(mae) + 1e-7


def test_cosine_full_size_sampled():
    """The paper's resolution 16 with 8 bands on a 2^22-query batch: a
    4096-query sample of S against the oracle."""
    R, B, J = 16, 8, 1 << 22
    qo = synth.sample_batch(synth.random_union(0), J, seed=1)
    p = band_params(R, B, seed=5)
    lb = lb32(R)
    S = api.efunc_cosine_forward(B, to_dev(p).reshape(-1), to_dev(qo), log_beta0=lb).cpu().numpy()
    idx = synth.rng(6).choice(J, 4096, replace=False)
    ref = oracle.cosine_forward(p, qo[idx, :3], R, B, log_beta0=lb)
    lim = S_tolerance(p, qo[idx, :3].astype(np.float64), R, B, lb)
    assert np.all(np.abs(S[idx] - ref) <= lim)


def test_cosine_forward_is_deterministic_and_order_independent():
    R, B, J = 8, 3, 30000
    p = to_dev(band_params(R, B, seed=7)).reshape(-1)
    qo = mixed_queries(R, J, seed=7)
    a = api.efunc_cosine_forward(B, p, to_dev(qo)).cpu().numpy()
    b = api.efunc_cosine_forward(B, p, to_dev(qo)).cpu().numpy()
    perm = synth.rng(3).permutation(J)
    c = api.efunc_cosine_forward(B, p, to_dev(qo[perm])).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a[perm], c)


@pytest.mark.parametrize("R", [1, 2, 3])
def test_cosine_tiny_grids(R):
    """Grids of 1, 2 or 3 centres per axis, where every window is clipped on
    at least one side: S and the gradient of 3 bands against the oracle."""
    B, J = 3, 3001
    p = band_params(R, B, seed=40 + R)
    qo = mixed_queries(R, J, seed=50 + R)
    lb = lb32(R)
    pd = to_dev(p).reshape(-1)
    S = api.efunc_cosine_forward(B, pd, to_dev(qo), log_beta0=lb).cpu().numpy()
    ref = oracle.cosine_forward(p, qo[:, :3], R, B, log_beta0=lb)
    lim = S_tolerance(p, qo[:, :3].astype(np.float64), R, B, lb)
    bad = np.flatnonzero(~(np.abs(S.astype(np.float64) - ref) <= lim))
    assert bad.size == 0, f"R={R}: {bad.size} of {J}; idx {bad[:5]} gpu {S[bad[:5]]} ref {ref[bad[:5]]}"
    gS = (synth.rng(60 + R).standard_normal(J) / J).astype(np.float32)
    grad = api.efunc_cosine_backward(B, pd, to_dev(qo), to_dev(gS), log_beta0=lb)
    g_ref = oracle.cosine_backward(p, qo[:, :3], gS, R, B, log_beta0=lb)
    b_floor = None
    if R == 1:
        # one key per band: softmax 1, O_b = f_b and dS/db_b = 0 exactly; the
        # kernel's value is gS w_b beta |q - key|^2 (f_b - O_b) per query with
        # f_b - O_b the rounding of f_b (2 x 4u |terms|) and of O_b = (l f) / l
        q = qo[:, :3].astype(np.float64)
        d2 = np.sum(q ** 2, axis=1)   # the one centre sits at the origin
        b_floor = []
        for b in range(B):
            w = np.prod(np.cos(b * np.pi * q), axis=1)
            o, d = p[b, 0, 1].astype(np.float64), p[b, 0, 2:].astype(np.float64)
            terms = np.abs(o) + np.abs(q * d).sum(axis=1)
            beta = np.exp(lb + np.float64(p[b, 0, 0]))
            b_floor.append(1.01 * np.sum(np.abs(gS * w) * beta * d2 * (8 * U32 * terms + 4 * U32 * terms)))
    assert_cosine_grad_close(grad.cpu().numpy(), g_ref, f"R={R}", b_floor=b_floor)


def test_cosine_empty_and_single_query():
    """An empty batch returns an empty S and leaves the gradient untouched;
    a single query (one sparse work item) matches the oracle."""
    R, B = 4, 5
    p = band_params(R, B, seed=70)
    pd = to_dev(p).reshape(-1)
    lb = lb32(R)
    empty = torch.zeros((0, 4), device=DEV)
    assert api.efunc_cosine_forward(B, pd, empty, log_beta0=lb).numel() == 0
    grad = torch.full_like(pd, 0.25)
    api.efunc_cosine_backward(B, pd, empty, torch.zeros(0, device=DEV), grad=grad, log_beta0=lb)
    assert torch.all(grad == 0.25)
    q = np.array([[0.1, -0.2, 0.3, 0.0]], np.float32)
    S = api.efunc_cosine_forward(B, pd, to_dev(q), log_beta0=lb).cpu().numpy()
    ref = oracle.cosine_forward(p, q[:, :3], R, B, log_beta0=lb)
    assert np.all(np.abs(S - ref) <= S_tolerance(p, q[:, :3].astype(np.float64), R, B, lb))
    gS = np.array([0.5], np.float32)
    grad = api.efunc_cosine_backward(B, pd, to_dev(q), to_dev(gS), log_beta0=lb)
    assert_cosine_grad_close(grad.cpu().numpy(), oracle.cosine_backward(p, q[:, :3], gS, R, B, log_beta0=lb),
                             "single query")


def test_cosine_fit_steps_match_oracle_trajectory():
    """Five MSE Adam steps of 3 bands against the oracle's loop (forward,
    loss gradient, backward, Adam per step); parameters agree wherever the
    first moment is far from zero."""
    R, B, J = 4, 3, 4000
    qo = synth.sample_batch(synth.sphere(0.5), J, seed=5)
    lb = lb32(R)
    p0 = (synth.rng(1).standard_normal((B, R ** 3, 5)) * 1e-3).astype(np.float32)
    pd, m, v = to_dev(p0).reshape(-1), torch.zeros(p0.size, device=DEV), torch.zeros(p0.size, device=DEV)
    stats = torch.zeros(10, device=DEV)
    api.efunc_cosine_fit(B, pd, m, v, to_dev(qo), steps=5, loss="mse", stats=stats, lr=1e-3, log_beta0=lb)
    pr, mr, vr = p0.astype(np.float64).reshape(-1), np.zeros(p0.size), np.zeros(p0.size)
    losses = []
    for step in range(1, 6):
        S = oracle.cosine_forward(pr.reshape(p0.shape), qo[:, :3], R, B, log_beta0=lb)
        gS, L, _ = oracle.loss_grad(S, qo[:, 3].astype(np.float64), oracle.MSE)
        g = oracle.cosine_backward(pr.reshape(p0.shape), qo[:, :3], gS, R, B, log_beta0=lb)
        pr, mr, vr = oracle.adam(pr, g.reshape(-1), mr, vr, step, lr=1e-3)
        losses.append(L)
    s = stats.cpu().numpy().reshape(5, 2)
    np.testing.assert_allclose(s[:, 0], losses, rtol=1e-4)
    solid = np.abs(mr) > 1e-3 * np.abs(mr).max()
    np.testing.assert_allclose(pd.cpu().numpy()[solid], pr[solid], rtol=1e-4, atol=1e-6)
