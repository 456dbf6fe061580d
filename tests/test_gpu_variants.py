"""GPU parity of the ablation variants (Table tab:ablation) through the C ABI
against the FP64 oracle's variant functions.

Tolerances (FP32 kernels vs FP64 oracle):
  forward O       |gpu - ref| <= max(1e-6 + 1e-5 |ref|, 4 u kappa + (nv + 3) u fabs)
                  kappa as for the default model (rounding of exponents and
                  weights); fabs = sum softmax * sum_m |term m of f|: the value
                  polynomial is summed term by term in FP32, each monomial up to
                  3 roundings, so f carries up to (nv + 3) u fabs of its own error
  dL/dparams      per channel group (offsets, log-scales, o, d, S, T of each
                  key set): max |gpu - ref| <= 1e-4 max |ref| of the group
Parameters are shaped like fitted grids (SDF value and gradient at each key,
random second / third order terms) unless stated; queries include cell-face
ties and points up to 0.6 outside the domain.
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
NV = [1, 4, 10, 20]
CONFIGS = ["G-1", "G-2", "G-3", "G-4", "G-5", "G-6", "G-7", "G-8", "Full-1", "Full-3"]


def groups(sets, deg, learn):
    """Channel groups (name -> columns) of a variant's parameter row."""
    out, base = {}, 0
    if sets & 2:
        out["Delta"] = [0, 1, 2]
        base = 3
    names = [n for s, n in ((1, "grid"), (2, "offset")) if sets & s]
    if learn:
        for i, n in enumerate(names):
            out[f"b {n}"] = [base + i]
        base += len(names)
    nv = NV[deg]
    for i, n in enumerate(names):
        o = base + i * nv
        out[f"o {n}"] = [o]
        if deg >= 1:
            out[f"d {n}"] = list(range(o + 1, o + 4))
        if deg >= 2:
            out[f"S {n}"] = list(range(o + 4, o + 10))
        if deg >= 3:
            out[f"T {n}"] = list(range(o + 10, o + 20))
    return out


def assert_variant_grad_close(gpu, ref, var, what, rtol=1e-4, floors=None):
    """floors: group name -> absolute bound added to the relative one (for a
    group whose exact gradient vanishes and whose kernel value is rounding)."""
    ch = ref.shape[1]
    gpu = np.asarray(gpu, dtype=np.float64).reshape(-1, ch)
    for name, cols in groups(*var).items():
        scale = np.abs(ref[:, cols]).max()
        err = np.abs(gpu[:, cols] - ref[:, cols]).max()
        floor = (floors or {}).get(name, 0.0)
        assert err <= rtol * scale + floor + 1e-30, f"{what} {name}: max err {err:.3e} vs scale {scale:.3e}"


def lone_key_scale_bound(gO, q, beta, f, fabs, nv):
    """Bound on the log-scale gradient when every query sees one key (R = 1,
    one key set): the softmax is 1, O = f and the exact dO/db is 0; the
    kernel's value is beta |q - key|^2 (f - O) per query, with f - O the
    rounding of f (evaluated in FP32, (nv + 3) u fabs on each of the forward
    and backward evaluations) and of O = (l f) / l (2u |f|), weight 1 + O(u)."""
    d2 = np.sum(np.asarray(q, np.float64) ** 2, axis=1)   # the one centre sits at the origin
    return 1.01 * np.sum(np.abs(gO) * beta * d2 * (2 * (nv + 3) * U32 * fabs + 4 * U32 * np.abs(f)))


def variant_tol(ref, kappa, fabs, deg):
    return np.maximum(1e-6 + 1e-5 * np.abs(ref), 4 * U32 * kappa + (NV[deg] + 3) * U32 * fabs)


def make_params(var, R, seed, shaped=True):
    shape = synth.random_union(seed) if shaped else None
    return synth.variant_params(shape, R, *var, seed=seed)


def test_variant_table_matches_the_paper_columns():
    """The named configurations: channel counts of Table tab:ablation."""
    expect = {"G-1": 1, "G-2": 4, "G-3": 10, "G-4": 20, "G-5": 2, "G-6": 5, "G-7": 11, "G-8": 21, "Full-1": 8,
              "Full-3": 13}
    for name, ch in expect.items():
        assert api.variant_channels(name) == ch == oracle.variant_channels(*api.VARIANTS[name])


@pytest.mark.parametrize("name", CONFIGS)
@pytest.mark.parametrize("R,J", [(4, 3001), (16, 40000)])
def test_variant_forward_matches_oracle(name, R, J):
    var = api.VARIANTS[name]
    p = make_params(var, R, seed=R + len(name))
    qo = mixed_queries(R, J, seed=3 * R)
    O = api.efunc_variant_forward(name, to_dev(p).reshape(-1), to_dev(qo), log_beta0=lb32(R)).cpu().numpy()
    ref, _, kap, fab = oracle.variant_forward(p, qo[:, :3], R, *var, log_beta0=lb32(R), want_diag=True)
    err = np.abs(O.astype(np.float64) - ref)
    lim = variant_tol(ref, kap, fab, var[1])
    bad = np.flatnonzero(~(err <= lim))
    assert bad.size == 0, (f"{name} R={R}: {bad.size} of {J} outside; idx {bad[:5]} gpu {O[bad[:5]]} "
                           f"ref {ref[bad[:5]]} lim {lim[bad[:5]]}")


@pytest.mark.parametrize("sets", [1, 2, 3])
@pytest.mark.parametrize("deg", [0, 1, 2, 3])
@pytest.mark.parametrize("learn", [0, 1])
def test_every_variant_forward_and_backward(sets, deg, learn):
    """All 24 (key sets, degree, scale) combinations at R = 5 (ragged
    boundary windows everywhere) with rough random parameters."""
    var = (sets, deg, learn)
    R, J = 5, 4001
    p = make_params(var, R, seed=sets + 4 * deg + 16 * learn, shaped=False)
    qo = mixed_queries(R, J, seed=sets + deg)
    pd = to_dev(p).reshape(-1)
    O = api.efunc_variant_forward(var, pd, to_dev(qo), log_beta0=lb32(R)).cpu().numpy()
    ref, _, kap, fab = oracle.variant_forward(p, qo[:, :3], R, *var, log_beta0=lb32(R), want_diag=True)
    err = np.abs(O.astype(np.float64) - ref)
    assert np.all(err <= variant_tol(ref, kap, fab, deg)), (var, err.max())
    gO = (synth.rng(9).standard_normal(J) / J).astype(np.float32)
    grad = api.efunc_variant_backward(var, pd, to_dev(qo), to_dev(gO), log_beta0=lb32(R))
    g_ref = oracle.variant_backward(p, qo[:, :3], gO, R, *var, log_beta0=lb32(R))
    assert_variant_grad_close(grad.cpu().numpy(), g_ref, var, f"{var}")


@pytest.mark.parametrize("name", ["G-6", "G-7", "G-8", "Full-1", "Full-3"])
@pytest.mark.parametrize("R,J", [(8, 20000), (32, 60000)])
def test_variant_backward_matches_oracle(name, R, J):
    var = api.VARIANTS[name]
    p = make_params(var, R, seed=2 * R)
    qo = mixed_queries(R, J, seed=5 * R)
    gO = (synth.rng(R).standard_normal(J) / J).astype(np.float32)
    grad = api.efunc_variant_backward(name, to_dev(p).reshape(-1), to_dev(qo), to_dev(gO), log_beta0=lb32(R))
    g_ref = oracle.variant_backward(p, qo[:, :3], gO, R, *var, log_beta0=lb32(R))
    assert_variant_grad_close(grad.cpu().numpy(), g_ref, var, f"{name} R={R}")


def test_variant_full3_agrees_with_the_default_model():
    """Full-3 is the default 13-float model: the variant kernels and the
    specialised fused kernels agree within both of their oracle tolerances."""
    R, J = 16, 30000
    p = synth.sdf_params(synth.random_union(2), R, seed=2)
    qo = mixed_queries(R, J, seed=8)
    lb = lb32(R)
    Ov = api.efunc_variant_forward("Full-3", to_dev(p).reshape(-1), to_dev(qo), log_beta0=lb).cpu().numpy()
    Od = api.efunc_forward(to_dev(p).reshape(-1), to_dev(qo), log_beta0=lb).cpu().numpy()
    ref, _, kap = oracle.forward(p.astype(np.float64), qo[:, :3].astype(np.float64), R, 2, lb, want_kappa=True)
    lim = np.maximum(1e-6 + 1e-5 * np.abs(ref), 4 * U32 * kap)
    assert np.all(np.abs(Ov - Od) <= 2 * lim)


@pytest.mark.parametrize("name", ["G-6", "G-8", "Full-1"])
@pytest.mark.parametrize("loss", ["l1", "mse"])
def test_variant_fit_step_gradient_and_loss(name, loss):
    """One fused variant step with lr = 0: Adam's first moment exposes the
    gradient (m = (1 - beta1) g); stats hold loss and MAE.  L1 targets sit at
    least 1e-3 from the oracle's O so both sides take the same sign."""
    var = api.VARIANTS[name]
    R, J = 16, 50000
    p = make_params(var, R, seed=11)
    qo = mixed_queries(R, J, seed=12)
    O_ref, _ = oracle.variant_forward(p, qo[:, :3], R, *var, log_beta0=lb32(R))
    g = synth.rng(13)
    qo[:, 3] = (O_ref + g.uniform(1e-3, 0.1, J) * np.where(g.integers(0, 2, J) == 0, -1.0, 1.0)).astype(np.float32)
    n = p.size
    pd, m, v = to_dev(p).reshape(-1), torch.zeros(n, device=DEV), torch.zeros(n, device=DEV)
    stats = torch.zeros(2, device=DEV)
    api.efunc_variant_fit(name, pd, m, v, to_dev(qo), steps=1, loss=loss, stats=stats, lr=0.0, log_beta0=lb32(R))
    gO, L, mae = oracle.loss_grad(O_ref, qo[:, 3].astype(np.float64), oracle.L1 if loss == "l1" else oracle.MSE)
    g_ref = oracle.variant_backward(p, qo[:, :3], gO, R, *var, log_beta0=lb32(R))
    assert_variant_grad_close(m.cpu().numpy() / 0.1, g_ref, var, f"{name} fit {loss}")
    np.testing.assert_array_equal(pd.cpu().numpy(), p.reshape(-1))
    s = stats.cpu().numpy()
    assert abs(s[0] - L) <= 1e-5 * abs(L) + 1e-7
    assert abs(s[1] - mae) <= 1e-5 * abs(mae) + 1e-7


def test_variant_fit_steps_match_oracle_trajectory():
    """Five MSE Adam steps of G-7 (degree-2 values) against the oracle's
    loop; parameters agree wherever the first moment is far from zero."""
    name = "G-7"
    var = api.VARIANTS[name]
    R, J = 4, 4000
    qo = synth.sample_batch(synth.sphere(0.5), J, seed=3)
    ch = api.variant_channels(name)
    p0 = (synth.rng(0).standard_normal((R ** 3, ch)) * 1e-3).astype(np.float32)
    pd, m, v = to_dev(p0).reshape(-1), torch.zeros(p0.size, device=DEV), torch.zeros(p0.size, device=DEV)
    stats = torch.zeros(10, device=DEV)
    api.efunc_variant_fit(name, pd, m, v, to_dev(qo), steps=5, loss="mse", stats=stats, lr=1e-3, log_beta0=lb32(R))
    pr, mr, vr = p0.astype(np.float64), np.zeros(p0.shape), np.zeros(p0.shape)
    losses = []
    for step in range(1, 6):
        O, _ = oracle.variant_forward(pr, qo[:, :3], R, *var, log_beta0=lb32(R))
        gO, L, _ = oracle.loss_grad(O, qo[:, 3].astype(np.float64), oracle.MSE)
        g = oracle.variant_backward(pr, qo[:, :3], gO, R, *var, log_beta0=lb32(R))
        pr, mr, vr = oracle.adam(pr.reshape(-1), g.reshape(-1), mr.reshape(-1), vr.reshape(-1), step, lr=1e-3)
        pr, mr, vr = pr.reshape(p0.shape), mr.reshape(p0.shape), vr.reshape(p0.shape)
        losses.append(L)
    s = stats.cpu().numpy().reshape(5, 2)
    np.testing.assert_allclose(s[:, 0], losses, rtol=1e-4)
    solid = np.abs(mr.reshape(-1)) > 1e-3 * np.abs(mr).max()
    np.testing.assert_allclose(pd.cpu().numpy()[solid], pr.reshape(-1)[solid], rtol=1e-4, atol=1e-6)


def test_variant_full_size_sampled():
    """G-6 and Full-1 at R = 32 with 2^22 queries (the benchmark's batch
    size): a 4096-query sample of the forward against the oracle."""
    R, J = 32, 1 << 22
    shape = synth.random_union(0)
    qo = synth.sample_batch(shape, J, seed=1)
    idx = synth.rng(2).choice(J, 4096, replace=False)
    for name in ("G-6", "Full-1"):
        var = api.VARIANTS[name]
        p = make_params(var, R, seed=3)
        O = api.efunc_variant_forward(name, to_dev(p).reshape(-1), to_dev(qo), log_beta0=lb32(R)).cpu().numpy()
        ref, _, kap, fab = oracle.variant_forward(p, qo[idx, :3], R, *var, log_beta0=lb32(R), want_diag=True)
        assert np.all(np.abs(O[idx] - ref) <= variant_tol(ref, kap, fab, var[1])), name


def test_variant_empty_and_single_query():
    R = 4
    var = api.VARIANTS["G-8"]
    p = make_params(var, R, seed=1)
    pd = to_dev(p).reshape(-1)
    assert api.efunc_variant_forward("G-8", pd, torch.zeros((0, 4), device=DEV)).numel() == 0
    q = np.array([[0.1, -0.2, 0.3, 0.0]], np.float32)
    O = api.efunc_variant_forward("G-8", pd, to_dev(q), log_beta0=lb32(R)).cpu().numpy()
    ref, _, kap, fab = oracle.variant_forward(p, q[:, :3], R, *var, log_beta0=lb32(R), want_diag=True)
    assert np.all(np.abs(O - ref) <= variant_tol(ref, kap, fab, 3))


@pytest.mark.parametrize("name", ["G-6", "G-8", "Full-3"])
def test_variant_forward_is_deterministic_and_order_independent(name):
    """Four summation classes combined in a fixed tree: a query's O does not
    depend on how many lanes share it or on the batch order (G-6 takes the
    lattice path in full windows, G-8 and Full-3 the generic one)."""
    var = api.VARIANTS[name]
    R, J = 8, 30000
    p = to_dev(make_params(var, R, seed=4)).reshape(-1)
    qo = mixed_queries(R, J, seed=6)
    a = api.efunc_variant_forward(name, p, to_dev(qo)).cpu().numpy()
    b = api.efunc_variant_forward(name, p, to_dev(qo)).cpu().numpy()
    perm = synth.rng(2).permutation(J)
    c = api.efunc_variant_forward(name, p, to_dev(qo[perm])).cpu().numpy()
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(a[perm], c)


@pytest.mark.parametrize("name", ["G-6", "G-8", "Full-3"])
@pytest.mark.parametrize("R", [1, 2, 3])
def test_variant_tiny_grids(name, R):
    """Grids of 1, 2 or 3 centres per axis (every window clipped): forward
    and backward against the oracle."""
    var = api.VARIANTS[name]
    J = 3001
    p = make_params(var, R, seed=20 + R)
    qo = mixed_queries(R, J, seed=30 + R)
    lb = lb32(R)
    pd = to_dev(p).reshape(-1)
    O = api.efunc_variant_forward(name, pd, to_dev(qo), log_beta0=lb).cpu().numpy()
    ref, _, kap, fab = oracle.variant_forward(p, qo[:, :3], R, *var, log_beta0=lb, want_diag=True)
    bad = np.flatnonzero(~(np.abs(O - ref) <= variant_tol(ref, kap, fab, var[1])))
    assert bad.size == 0, f"{name} R={R}: {bad.size} of {J}; idx {bad[:5]} gpu {O[bad[:5]]} ref {ref[bad[:5]]}"
    gO = (synth.rng(R).standard_normal(J) / J).astype(np.float32)
    grad = api.efunc_variant_backward(name, pd, to_dev(qo), to_dev(gO), log_beta0=lb)
    g_ref = oracle.variant_backward(p, qo[:, :3], gO, R, *var, log_beta0=lb)
    floors = None
    if R == 1 and var[0] == 1:   # one key per query: dO/db vanishes
        beta = np.exp(lb + np.float64(p[0, 0]))
        floors = {"b grid": lone_key_scale_bound(gO, qo[:, :3], beta, ref, fab, NV[var[1]])}
    assert_variant_grad_close(grad.cpu().numpy(), g_ref, var, f"{name} R={R}", floors=floors)
