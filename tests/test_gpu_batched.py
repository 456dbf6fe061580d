"""The batched fit of many shapes (efunc_fit_batched, efunc_eval_batched,
efunc_tune_batched) against the oracle and against the single-shape calls.

Every shape of a batched launch must get exactly what it would get alone:
its gradient (per slot type within 1e-4 of the slot's largest |ref|, FP32
atomics), its loss statistics (1e-5), its Adam trajectory.  Shapes of
different resolutions and uneven query counts share one sort, one key pack,
one fused launch and one Adam step per step.
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

RS = [1, 3, 8, 16, 5, 32]
JS = [500, 3001, 20011, 4097, 777, 60000]


def lb32(R):
    return float(np.float32(oracle.default_log_beta0(R)))


def batch_rows(b, seed):
    return np.concatenate([synth.sample_batch(synth.random_union(seed + s), J, seed=seed * 100 + s)
                           for s, J in enumerate(b.Js)])


def batch_params(b, seed, kind="sdf"):
    parts = []
    for s, R in enumerate(b.Rs):
        parts.append((synth.sdf_params(synth.random_union(seed + s), R, seed=seed + s) if kind == "sdf"
                      else synth.init_params(R, seed=seed + s)).reshape(-1))
    return np.concatenate(parts).astype(np.float32)


U32 = 2.0 ** -24


def assert_grad_close(gpu, ref, what, rtol=1e-4, terms=None):
    """Per slot type rtol * max|ref| plus the entry's own rounding bound from
    the oracle's error terms (as in test_gpu_parity.py)."""
    gpu = np.asarray(gpu, dtype=np.float64).reshape(-1, 13)
    ref = ref.reshape(-1, 13)
    extra = np.zeros_like(ref) if terms is None else (8 * U32 * terms[1] + 6 * U32 * terms[0]).reshape(-1, 13)
    for name, cols in SLOT_TYPES.items():
        scale = np.abs(ref[:, cols]).max()
        err = np.abs(gpu[:, cols] - ref[:, cols])
        lim = rtol * scale + 1e-30 + extra[:, cols]
        margins.record(f"{what} [{name}]", err, lim)
        assert np.all(err <= lim), f"{what} slot {name}: max err {err.max():.3e} vs scale {scale:.3e}"


def test_batched_step_matches_oracle_per_shape():
    """One batched MSE step with lr = 0: Adam's first moment is (1 - beta1) g
    for every shape's grid; the per-shape (loss, MAE) statistics and
    gradients equal the oracle's for that shape alone."""
    b = api.Batch(RS, JS)
    p = batch_params(b, 1)
    rows = batch_rows(b, 1)
    pd = torch.from_numpy(p).to(DEV)
    m, v = torch.zeros_like(pd), torch.zeros_like(pd)
    stats = torch.zeros(b.S * 2, device=DEV)
    b.fit(pd, m, v, torch.from_numpy(rows).to(DEV), steps=1, loss="mse", stats=stats, lr=0.0)
    st = stats.view(b.S, 2).cpu().numpy()
    mm = m.cpu().numpy() / 0.1
    for s, (R, J) in enumerate(zip(b.Rs, b.Js)):
        ps = p[b.param_offsets[s]:b.param_offsets[s + 1]].astype(np.float64)
        qs = rows[b.query_offsets[s]:b.query_offsets[s + 1]].astype(np.float64)
        O, _ = oracle.forward(ps, qs, R, 2, lb32(R))
        gO, L, mae = oracle.loss_grad(O, qs[:, 3], oracle.MSE)
        g_ref = oracle.backward(ps, qs, gO, R, 2, lb32(R))
        assert_grad_close(mm[b.param_offsets[s]:b.param_offsets[s + 1]], g_ref, f"batched shape {s} R={R}",
                          terms=oracle.backward_error_terms(ps, qs, gO, R, 2, lb32(R)))
        assert abs(st[s, 0] - L) <= 1e-5 * L + 1e-9 and abs(st[s, 1] - mae) <= 1e-5 * mae + 1e-9
    np.testing.assert_array_equal(pd.cpu().numpy(), p)


@pytest.mark.parametrize("graph", [False, True])
def test_batched_trajectory_matches_single_shape_fits(graph):
    """Seven Adam steps over two batches: every shape's losses and parameters
    follow its own single-shape efunc_fit on the same batch sequence (the
    parameters wherever the first moment is far from zero)."""
    b = api.Batch(RS[:5], JS[:5])
    p0 = batch_params(b, 2, kind="init")
    r0, r1 = batch_rows(b, 3), batch_rows(b, 4)
    qo = torch.from_numpy(np.concatenate([r0, r1])).to(DEV)
    pd = torch.from_numpy(p0).to(DEV)
    m, v = torch.zeros_like(pd), torch.zeros_like(pd)
    steps = 7
    stats = torch.zeros(steps * b.S * 2, device=DEV)
    b.fit(pd, m, v, qo, steps=steps, n_batches=2, loss="mse", stats=stats, lr=1e-3, graph=graph)
    st = stats.view(steps, b.S, 2).cpu().numpy()
    for s, (R, J) in enumerate(zip(b.Rs, b.Js)):
        sl = slice(b.param_offsets[s], b.param_offsets[s + 1])
        q_s = torch.from_numpy(np.concatenate([r0[b.query_offsets[s]:b.query_offsets[s + 1]],
                                               r1[b.query_offsets[s]:b.query_offsets[s + 1]]])).to(DEV)
        ps = torch.from_numpy(p0[sl].copy()).to(DEV)
        ms_, vs_ = torch.zeros_like(ps), torch.zeros_like(ps)
        ss = torch.zeros(2 * steps, device=DEV)
        api.efunc_fit(ps, ms_, vs_, q_s, steps=steps, J=J, n_batches=2, loss="mse", stats=ss, lr=1e-3,
                      log_beta0=lb32(R), ws=api.Workspace(DEV))
        np.testing.assert_allclose(st[:, s, :], ss.view(steps, 2).cpu().numpy(), rtol=1e-5)
        mref = ms_.cpu().numpy()
        solid = np.abs(mref) > 1e-2 * np.abs(mref).max()
        np.testing.assert_allclose(pd.cpu().numpy()[sl][solid], ps.cpu().numpy()[solid], rtol=1e-4, atol=1e-6)


def test_batched_eval_matches_single_shape_eval():
    b = api.Batch(RS, JS)
    p = torch.from_numpy(batch_params(b, 5)).to(DEV)
    rows = torch.from_numpy(batch_rows(b, 6)).to(DEV)
    out = b.eval(p, rows).cpu().numpy()
    for s, R in enumerate(b.Rs):
        ref = api.efunc_eval_loss(b.params_of(p, s).contiguous(), b.rows_of(rows, s).contiguous(),
                                  log_beta0=lb32(R)).cpu().numpy()
        np.testing.assert_allclose(out[s], ref, rtol=1e-6)


def test_tuning_knobs_give_the_same_fit():
    """A non-default launch configuration (128-query items, other lane
    thresholds, 2 sort blocks per SM) takes the same steps."""
    b = api.Batch(RS, JS)
    p0 = batch_params(b, 7, kind="init")
    qo = torch.from_numpy(batch_rows(b, 8)).to(DEV)
    out = []
    for tune in (None, (128, 96, 48, 2)):
        b.tuning = None if tune is None else api.B.Tuning(*tune)
        pd = torch.from_numpy(p0).to(DEV)
        m, v = torch.zeros_like(pd), torch.zeros_like(pd)
        stats = torch.zeros(3 * b.S * 2, device=DEV)
        b.fit(pd, m, v, qo, steps=3, loss="mse", stats=stats, lr=1e-3)
        out.append((pd.cpu().numpy(), m.cpu().numpy(), stats.cpu().numpy()))
    np.testing.assert_allclose(out[1][2], out[0][2], rtol=1e-5)
    solid = np.abs(out[0][1]) > 1e-2 * np.abs(out[0][1]).max()
    np.testing.assert_allclose(out[1][0][solid], out[0][0][solid], rtol=1e-4, atol=1e-6)


def test_tuner_picks_a_valid_configuration_and_leaves_the_fit_state():
    b = api.Batch(RS, JS)
    p0 = batch_params(b, 9)
    pd = torch.from_numpy(p0).to(DEV)
    m, v = torch.ones_like(pd), torch.ones_like(pd)
    cfg, ms = b.tune(pd, m, v, torch.from_numpy(batch_rows(b, 10)).to(DEV), trial_steps=2)
    assert cfg["chunk"] in (128, 256) and cfg["sort_blocks"] in (4, 8) and cfg["group_max"] in (0, 64, 128)
    assert ms > 0
    np.testing.assert_array_equal(pd.cpu().numpy(), p0)
    assert m.abs().max().item() == 0.0 and v.abs().max().item() == 0.0
