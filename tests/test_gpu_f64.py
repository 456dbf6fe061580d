"""The FP64 instantiation of the fused kernels (efunc_forward_f64 /
efunc_backward_f64) and torch.autograd.gradcheck of EfuncFn through it.

The FP64 kernels are the FP32 hot-path kernels compiled for double (same
staging, window choice from FP32-rounded coordinates, summation classes and
branches; exp2 / log2 in double instead of the SFU approximations).  Against
the FP64 oracle they agree to rounding: |gpu - ref| <= 1e-12 + 1e-11 |ref| +
2^-46 kappa for O (kappa as in the FP32 tests: the sum order and exp2 vs exp
perturb each exponent by a few FP64 ulps), per slot type 1e-10 max |ref| for
the gradients.  gradcheck then compares the FP64 kernels' analytical
Jacobian (Algorithm 2, Eq. func-normal) with central finite differences of
the FP64 forward, on an 8^3 grid with 256 queries kept 1 % of a cell away
from every window boundary (the windowed model is discontinuous there).
"""
import numpy as np
import pytest
import torch

import margins
import oracle
from paper_2505_21319_gb300 import api, synth

pytestmark = pytest.mark.gpu
DEV = "cuda"
SLOT_TYPES = {"Delta": [0, 1, 2], "b": [3], "b'": [4], "o": [5], "d": [6, 7, 8], "o'": [9], "d'": [10, 11, 12]}
U64 = 2.0 ** -52


def lb32(R):
    return float(np.float32(oracle.default_log_beta0(R)))


def queries(R, J, seed, outside=True):
    g = synth.rng(seed)
    q = synth.sample_batch(synth.random_union(seed), J, seed=seed)[:, :3].astype(np.float64)
    q += g.normal(0, 1e-3, q.shape)   # FP64 coordinates that FP32 does not represent
    if outside:
        n_out = J // 16
        q[:n_out] = g.uniform(-1.5, 1.5, (n_out, 3))
    return q


@pytest.mark.parametrize("R,J,pkind", [(1, 500, "random"), (2, 1000, "random"), (8, 20011, "random"),
                                       (16, 30000, "sdf"), (32, 40000, "sdf")])
def test_f64_forward_and_backward_match_oracle(R, J, pkind):
    q = queries(R, J, seed=R)
    p = (synth.random_params(R, seed=R) if pkind == "random"
         else synth.sdf_params(synth.random_union(R), R, seed=R)).astype(np.float64)
    lb = lb32(R)
    pd, qd = torch.from_numpy(p).to(DEV), torch.from_numpy(q).to(DEV)
    O, lse, dq = api.efunc_forward_f64(pd, qd, log_beta0=lb, want_lse=True, want_dq=True)
    O_ref, lse_ref, dq_ref, kappa, sens = oracle.forward(p, q, R, 2, lb, want_dq=True, want_kappa=True,
                                                         want_dq_sens=True)
    for name, got, ref, lim in (
            ("O", O, O_ref, 1e-12 + 1e-11 * np.abs(O_ref) + 64 * U64 * kappa),
            ("lse", lse, lse_ref, 1e-12 + 1e-11 * np.abs(lse_ref)),
            ("dO/dq", dq, dq_ref, 1e-10 * np.abs(dq_ref) + 1e-11 * np.abs(dq_ref).max()
             + (sens * 64 * U64 * kappa)[:, None])):
        err = np.abs(got.cpu().numpy() - ref)
        margins.record(f"f64 {name}", err, lim)
        assert np.all(err <= lim), f"{name}: worst {err.max():.3e}"
    gO = synth.rng(R + 1).standard_normal(J) / J
    grad, gq = api.efunc_backward_f64(pd, qd, torch.from_numpy(gO).to(DEV), want_gq=True, log_beta0=lb)
    g_ref, gq_ref = oracle.backward(p, q, gO, R, 2, lb, want_gq=True)
    grad = grad.cpu().numpy().reshape(-1, 13)
    g_ref = g_ref.reshape(-1, 13)
    for name, cols in SLOT_TYPES.items():
        scale = np.abs(g_ref[:, cols]).max()
        err = np.abs(grad[:, cols] - g_ref[:, cols]).max()
        margins.record(f"f64 grad [{name}]", err, 1e-10 * scale + 1e-300)
        assert err <= 1e-10 * scale + 1e-300, f"slot {name}: {err:.3e} vs {scale:.3e}"
    err = np.abs(gq.cpu().numpy() - gq_ref)
    assert err.max() <= 1e-10 * np.abs(gq_ref).max() + 1e-300


def test_f64_forward_is_independent_of_query_order():
    R, J = 8, 5000
    q = queries(R, J, seed=3)
    p = torch.from_numpy(synth.random_params(R, seed=3).astype(np.float64)).to(DEV)
    a = api.efunc_forward_f64(p, torch.from_numpy(q).to(DEV)).cpu().numpy()
    perm = synth.rng(4).permutation(J)
    b = api.efunc_forward_f64(p, torch.from_numpy(q[perm]).to(DEV)).cpu().numpy()
    np.testing.assert_array_equal(a[perm], b)


def _away_from_window_boundaries(R, J, seed):
    """Queries inside the domain at least 1 % of a cell from every plane
    through centres (where the window base index changes)."""
    g = synth.rng(seed)
    h = 2.0 / R
    out = []
    while len(out) < J:
        x = g.uniform(-1, 1, 3)
        u = (x + 1) / h - 0.5   # window base changes where u is an integer
        if np.all(np.abs(u - np.round(u)) > 0.01):
            out.append(x)
    return np.array(out)


def test_gradcheck_autograd_function_fp64():
    """torch.autograd.gradcheck of EfuncFn (params and query positions) on
    an 8^3 grid with 256 queries, in FP64 through the CUDA kernels."""
    R, J = 8, 256
    p = synth.sdf_params(synth.random_union(2), R, seed=2).astype(np.float64)
    q = _away_from_window_boundaries(R, J, seed=5)
    pd = torch.from_numpy(p).to(DEV).requires_grad_(True)
    qd = torch.from_numpy(q).to(DEV).requires_grad_(True)
    lb = lb32(R)
    # the gradient's double atomics are summed in arrival order: repeated
    # backward calls may differ by a few ulps (nondet_tol)
    assert torch.autograd.gradcheck(lambda a, b: api.EfuncFn.apply(a, b, lb), (pd, qd), eps=1e-6, atol=1e-7,
                                    rtol=1e-5, nondet_tol=1e-12)


def test_gradcheck_with_rough_parameters_and_window_queries():
    """The same check with every slot rough (random_params: offsets, scales
    and values far from zero), queries in every sort of window (grid corners
    and faces included), on a 4^3 grid."""
    R, J = 4, 128
    p = synth.random_params(R, seed=7).astype(np.float64)
    q = _away_from_window_boundaries(R, J, seed=8)
    q[:8] = np.array([[sx, sy, sz] for sx in (-0.97, 0.96) for sy in (-0.95, 0.98) for sz in (-0.99, 0.97)])
    pd = torch.from_numpy(p).to(DEV).requires_grad_(True)
    qd = torch.from_numpy(q).to(DEV).requires_grad_(True)
    lb = lb32(R)
    assert torch.autograd.gradcheck(lambda a, b: api.EfuncFn.apply(a, b, lb), (pd, qd), eps=1e-6, atol=1e-6,
                                    rtol=1e-5, nondet_tol=1e-12)


@pytest.mark.parametrize("R,J", [(4, 3001), (16, 65536), (32, 1 << 18)])
def test_eval_loss_matches_oracle(R, J):
    shape = synth.random_union(R)
    qo = synth.sample_batch(shape, J, seed=R + 2)
    p = synth.sdf_params(shape, R, seed=R)
    lb = lb32(R)
    out = api.efunc_eval_loss(torch.from_numpy(p).to(DEV), torch.from_numpy(qo).to(DEV), log_beta0=lb)
    O_ref, _ = oracle.forward(p.astype(np.float64), qo.astype(np.float64), R, 2, lb)
    d = O_ref - qo[:, 3].astype(np.float64)
    mse, mae = float((d ** 2).mean()), float(np.abs(d).mean())
    got = out.cpu().numpy().astype(np.float64)
    margins.record("eval mse", abs(got[0] - mse), 1e-5 * mse)
    margins.record("eval mae", abs(got[1] - mae), 1e-5 * mae)
    assert abs(got[0] - mse) <= 1e-5 * mse and abs(got[1] - mae) <= 1e-5 * mae
