"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these compares the oracle with itself: each check uses an invariant,
a closed-form special case, a library routine that the special case reduces
to, brute force, or finite differences.  A dropped term, a flipped sign, a
transposed index or a wrong key position in the oracle fails at least one.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.special
import scipy.spatial.distance
import torch

import oracle
from paper_2505_21319_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def centres(R):
    """Centre positions from the stated reading: -1 + (idx + 0.5) * 2/R, x slowest."""
    c = -1.0 + (np.arange(R) + 0.5) * (2.0 / R)
    a, b, d = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([a.ravel(), b.ravel(), d.ravel()], 1)


def queries(seed, J, spread=1.1):
    return synth.rng(seed).uniform(-spread, spread, size=(J, 3)).astype(np.float32).astype(np.float64)


def keys_of(params, R, log_beta0):
    """Explicit key list (positions, beta, o, d) for the whole grid."""
    p = np.asarray(params, dtype=np.float64).reshape(R ** 3, 13)
    k = centres(R)
    pos = np.concatenate([k, k + p[:, 0:3]])
    beta = np.exp(log_beta0 + np.concatenate([p[:, 3], p[:, 4]]))
    o = np.concatenate([p[:, 5], p[:, 9]])
    d = np.concatenate([p[:, 6:9], p[:, 10:13]])
    return pos, beta, o, d


# --------------------------------------------------------------- layout pins

def test_parameter_counts_match_paper():
    """Table tab:main / tab:ablation / Fig. comp-trilinear print the float
    counts of the representation; 13 floats per centre and I = R^3."""
    g = json.load(open(os.path.join(GOLDEN, "param_counts.json")))
    for row in g["table_main_ours"]:
        n = row["R"] ** 3 * oracle.NSLOT
        if "value" in row:
            assert n == row["value"]
        else:
            assert abs(n - row["approx"]) <= row["rel_tol"] * row["approx"]
    full = [r for r in g["table_ablation"] if r["floats_per_centre"] == 13]
    assert full and all(r["R"] ** 3 * oracle.NSLOT == r["value"] for r in full)
    for r in g["table_ablation"]:
        assert r["R"] ** 3 * r["floats_per_centre"] == r["value"]
    # Eq. func-offset: 5 + |phi| + |phi'| with first-order phi (1 + 3 floats)
    assert 5 + 4 + 4 == oracle.NSLOT


# --------------------------------------------------------------- value pins

@pytest.mark.parametrize("R,W", [(1, 1), (2, 2), (3, 1), (8, 2), (5, 5)])
def test_partition_of_unity(R, W):
    """Eq. nrbf: the normalised weights form a convex combination, so equal
    constant values reproduce that constant for any keys, scales, offsets."""
    p = synth.random_params(R, seed=R, delta_scale=0.8, b_scale=1.0).astype(np.float64)
    p[:, 5] = 0.375
    p[:, 9] = 0.375
    p[:, 6:9] = 0.0
    p[:, 10:13] = 0.0
    q = queries(11, 200)
    O, lse, dq = oracle.forward(p, q, R, W, want_dq=True)
    np.testing.assert_allclose(O, 0.375, rtol=0, atol=1e-14)
    np.testing.assert_allclose(dq, 0.0, atol=1e-9)


@pytest.mark.parametrize("R,W", [(1, 1), (2, 2), (4, 2), (8, 2), (3, 3)])
def test_affine_reproduction(R, W):
    """Shift-invariance of f (Sec. 3.2): if every key holds the same global
    affine function P(x) = a + b.x expressed about its own position, the blend
    is P(q) exactly and dO/dq = b (Eq. func-normal), whatever the weights."""
    rng = synth.rng(100 + R)
    a = 0.3
    b = np.array([0.7, -1.3, 0.45])
    p = synth.random_params(R, seed=7 * R, delta_scale=0.9, b_scale=1.0).astype(np.float64)
    k = centres(R)
    p[:, 5] = a + k @ b
    p[:, 6:9] = b
    p[:, 9] = a + (k + p[:, 0:3]) @ b
    p[:, 10:13] = b
    q = queries(12 + R, 300)
    O, _, dq = oracle.forward(p, q, R, W, want_dq=True)
    np.testing.assert_allclose(O, a + q @ b, rtol=0, atol=1e-13)
    np.testing.assert_allclose(dq, np.broadcast_to(b, dq.shape), rtol=0, atol=1e-10)
    # dO/d(log-scales) vanish because f - O == 0 for every key; dO/dDelta = -d' w + 0
    gO = rng.standard_normal(q.shape[0])
    g = oracle.backward(p, q, gO, R, W)
    np.testing.assert_allclose(g[:, 3:5], 0.0, atol=1e-10)


def test_two_key_logistic_closed_form():
    """R = 1: one centre, two keys (grid key at the origin, offset key at
    Delta).  With constant values the softmax over two keys is the logistic
    function of the exponent difference (Eq. nrbf):
        O = o' + (o - o') * expit(beta'|q - Delta|^2 - beta|q|^2)."""
    rng = synth.rng(5)
    for _ in range(20):
        th = np.zeros((1, 13))
        th[0, 0:3] = rng.uniform(-0.5, 0.5, 3)
        th[0, 3:5] = rng.uniform(-2, 2, 2)
        th[0, 5] = rng.uniform(-1, 1)
        th[0, 9] = rng.uniform(-1, 1)
        lb = rng.uniform(0, 3)
        q = rng.uniform(-1, 1, (5, 3)).astype(np.float32).astype(np.float64)
        beta, betap = math.exp(lb + th[0, 3]), math.exp(lb + th[0, 4])
        z = betap * ((q - th[0, 0:3]) ** 2).sum(1) - beta * (q ** 2).sum(1)
        want = th[0, 9] + (th[0, 5] - th[0, 9]) * scipy.special.expit(z)
        O, _ = oracle.forward(th, q, 1, 1, log_beta0=lb)
        np.testing.assert_allclose(O, want, rtol=1e-13, atol=1e-14)


def test_symmetric_midpoint_and_nearest_key_limit():
    """Two keys with equal scale: a query at their midpoint weighs them 1/2
    each.  With a very large scale the blend tends to the nearest key's value
    (the weight of every other key vanishes)."""
    th = np.zeros((1, 13))
    th[0, 0:3] = [0.4, -0.2, 0.1]
    th[0, 5], th[0, 9] = 2.0, -1.0
    mid = np.array([[0.2, -0.1, 0.05]])
    O, _ = oracle.forward(th, mid, 1, 1, log_beta0=1.0)
    assert abs(O[0] - 0.5) < 1e-15
    # the grid key sits at the origin: a query next to it, huge beta -> o
    O, _ = oracle.forward(th, np.array([[0.01, 0.0, 0.0]]), 1, 1, log_beta0=12.0)
    assert abs(O[0] - 2.0) < 1e-12
    O, _ = oracle.forward(th, np.array([[0.39, -0.2, 0.1]]), 1, 1, log_beta0=12.0)
    assert abs(O[0] + 1.0) < 1e-12


@pytest.mark.parametrize("R", [2, 3, 4])
def test_f0_reduces_to_nrbf_library_softmax(R):
    """Sec. 3.2: with zero linear terms (f^0) the model is the normalised RBF of
    Eq. nrbf.  Global support (W >= R) against scipy's softmax over the
    pairwise squared distances of all 2I keys."""
    lb = 2.5
    p = synth.random_params(R, seed=31 + R, delta_scale=0.7, b_scale=0.8).astype(np.float64)
    p[:, 6:9] = 0.0
    p[:, 10:13] = 0.0
    q = queries(3 + R, 64)
    pos, beta, o, _ = keys_of(p, R, lb)
    D2 = scipy.spatial.distance.cdist(q, pos, "sqeuclidean")
    want = scipy.special.softmax(-beta[None, :] * D2, axis=1) @ o
    O, lse = oracle.forward(p, q, R, W=R, log_beta0=lb)
    np.testing.assert_allclose(O, want, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(lse, scipy.special.logsumexp(-beta[None, :] * D2, axis=1), rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------- window pins

@pytest.mark.parametrize("R", [2, 3, 4, 5])
def test_window_at_least_R_equals_global_brute_force(R):
    """Brute force over all 2I keys (the paper's global Algorithm 1) equals the
    windowed oracle once the window covers the grid (W >= R)."""
    p = synth.random_params(R, seed=R, delta_scale=0.9, b_scale=0.7).astype(np.float64)
    q = queries(40 + R, 100, spread=1.3)
    O, _ = oracle.forward(p, q, R, W=R)
    G = oracle.forward_global(p, q, R)
    np.testing.assert_allclose(O, G, rtol=1e-12, atol=1e-13)


def test_window_truncation_error_bound():
    """W = 2 drops keys at least 2h away along some axis; with the initial scale
    (beta h^2 = 4e^7/1024) and no offsets every dropped key weighs at most
    exp(-beta h^2 (4 - 3/4)) of the nearest one, so |O_W - O_global| is bounded
    by 2I times that, times the spread of values."""
    R = 8
    p = synth.random_params(R, seed=9, delta_scale=0.0, b_scale=0.0).astype(np.float64)
    q = queries(77, 300, spread=1.0)
    O, _ = oracle.forward(p, q, R, W=2)
    G = oracle.forward_global(p, q, R)
    h = 2.0 / R
    bh2 = math.exp(oracle.default_log_beta0(R)) * h * h
    spread = np.abs(p[:, 5:13]).max() * 4.0
    bound = 2 * R ** 3 * math.exp(-bh2 * (4 - 0.75)) * spread
    assert np.abs(O - G).max() <= bound
    assert np.abs(O - G).max() > 0  # the window really truncates


def test_window_base_fp32_formula():
    """Window base c = clamp(floor((q+1)*R/2 - 1/2), -1, R-1): against exact
    rational arithmetic wherever FP32 rounding cannot move the floor, against
    numpy FP32 arithmetic everywhere (ties included), and its clamping."""
    from fractions import Fraction
    rng = synth.rng(3)
    for R in (1, 2, 7, 16, 32, 64):
        qs = list(rng.uniform(-1.2, 1.2, 400).astype(np.float32))
        # exact ties: cell-centre positions and grid faces
        qs += [np.float32(-1 + i / R) for i in range(0, 2 * R + 1)]
        qs += [np.nextafter(np.float32(-1 + i / R), np.float32(2)) for i in range(0, 2 * R + 1)]
        for q in qs:
            q = np.float32(q)
            c = oracle.window_base(float(q), R)
            u = (q + np.float32(1)) * np.float32(R * 0.5) - np.float32(0.5)
            c32 = int(np.floor(np.clip(u, np.float32(-1), np.float32(R - 1))))
            assert c == c32
            exact = Fraction(float(q)) * 0 + (Fraction(float(q)) + 1) * Fraction(R, 2) - Fraction(1, 2)
            fl = math.floor(exact)
            if abs(exact - fl) > Fraction(1, 1 << 18) and abs(exact - fl - 1) > Fraction(1, 1 << 18):
                assert c == max(-1, min(R - 1, fl))
    assert oracle.window_base(float("nan"), 8) == -1
    assert oracle.window_base(1e30, 8) == 7 and oracle.window_base(-1e30, 8) == -1


def test_window_contents_brute_force():
    """The window is the set of (2W)^3 centres whose index lies in
    [c - W + 1, c + W] per axis; verified by enumerating every centre on a tiny
    grid and zeroing the values of all centres outside that set: the output
    must not change, while changing a centre inside it must."""
    R, W = 6, 2
    p = synth.random_params(R, seed=4).astype(np.float64)
    q = queries(9, 30, spread=1.0)
    O, _ = oracle.forward(p, q, R, W)
    for j in range(q.shape[0]):
        c = [oracle.window_base(q[j, a], R) for a in range(3)]
        idx = np.arange(R ** 3)
        ia, ib, ic = idx // (R * R), (idx // R) % R, idx % R
        inside = np.ones(R ** 3, bool)
        for a, ii in enumerate((ia, ib, ic)):
            inside &= (ii >= c[a] - W + 1) & (ii <= c[a] + W)
        p2 = p.copy()
        p2[~inside, 5:13] = 123.0
        O2, _ = oracle.forward(p2, q[j:j + 1], R, W)
        assert O2[0] == O[j]
        ins = np.flatnonzero(inside)
        k = ins[np.argmin(((centres(R)[ins] - q[j]) ** 2).sum(1))]
        p3 = p.copy()
        p3[k, 5] += 1.0
        O3, _ = oracle.forward(p3, q[j:j + 1], R, W)
        assert O3[0] != O[j]


# --------------------------------------------------------- gradient pins

def _fd_params(p, q, gO, R, W, lb, entries, eps=1e-6):
    out = []
    for (i, s) in entries:
        hstep = eps * max(1.0, abs(p[i, s]))
        pp, pm = p.copy(), p.copy()
        pp[i, s] += hstep
        pm[i, s] -= hstep
        Op, _ = oracle.forward(pp, q, R, W, lb)
        Om, _ = oracle.forward(pm, q, R, W, lb)
        out.append(float(gO @ (Op - Om)) / (2 * hstep))
    return np.array(out)


@pytest.mark.parametrize("R,W", [(3, 3), (6, 2)])
def test_param_gradients_match_central_differences(R, W):
    """Algorithm 2 / Sec. 3.6 closed forms against FP64 central differences of
    L = sum_j gO_j O(q_j), for all 13 slots of the centres the queries touch.
    With W < R the queries stay 1e-3 h away from window switches, where the
    windowed model is smooth."""
    lb = oracle.default_log_beta0(R) - 1.0
    p = synth.random_params(R, seed=50 + R, delta_scale=0.6, b_scale=0.5).astype(np.float64)
    rng = synth.rng(60 + R)
    q = rng.uniform(-0.95, 0.95, (6, 3))
    if W < R:
        t = (q + 1) * R / 2 - 0.5
        frac = t - np.floor(t)
        q = np.where(np.minimum(frac, 1 - frac) < 1e-3, q + 0.01, q)
    q = q.astype(np.float32).astype(np.float64)
    gO = rng.standard_normal(q.shape[0])
    grad = oracle.backward(p, q, gO, R, W, lb)
    touched = np.flatnonzero(np.abs(grad).sum(1) > 0)
    assert touched.size > 0
    sel = rng.choice(touched, size=min(10, touched.size), replace=False)
    entries = [(i, s) for i in sel for s in range(13)]
    fd = _fd_params(p, q, gO, R, W, lb, entries)
    an = np.array([grad[i, s] for (i, s) in entries])
    scale = np.abs(an).max()
    np.testing.assert_allclose(an, fd, rtol=1e-6, atol=1e-7 * scale)
    # untouched centres get exactly zero
    assert np.all(grad[np.setdiff1d(np.arange(R ** 3), touched)] == 0.0)


@pytest.mark.parametrize("R,W", [(3, 3), (5, 2)])
def test_query_gradient_matches_central_differences(R, W):
    """Eq. func-normal against FP64 central differences in q (away from window
    switches), and dL/dq = gO * dO/dq from the backward."""
    lb = oracle.default_log_beta0(R) - 0.5
    p = synth.random_params(R, seed=70 + R, delta_scale=0.6, b_scale=0.5).astype(np.float64)
    rng = synth.rng(80 + R)
    q = rng.uniform(-0.9, 0.9, (8, 3))
    t = (q + 1) * R / 2 - 0.5
    frac = t - np.floor(t)
    q = np.where(np.minimum(frac, 1 - frac) < 1e-3, q + 0.01, q)
    _, _, dq = oracle.forward(p, q, R, W, lb, want_dq=True)
    eps = 1e-6
    for a in range(3):
        qp, qm = q.copy(), q.copy()
        qp[:, a] += eps
        qm[:, a] -= eps
        fd = (oracle.forward(p, qp, R, W, lb)[0] - oracle.forward(p, qm, R, W, lb)[0]) / (2 * eps)
        np.testing.assert_allclose(dq[:, a], fd, rtol=1e-6, atol=1e-7 * np.abs(fd).max())
    gO = rng.standard_normal(q.shape[0])
    _, gq = oracle.backward(p, q, gO, R, W, lb, want_gq=True)
    np.testing.assert_allclose(gq, gO[:, None] * dq, rtol=1e-14, atol=0)


def test_value_gradient_sums_to_one():
    """Partition of unity for the gradient: dO/do summed over all keys is
    sum_i softmax_i = 1 for every query, so with gO = 1 for one query the
    o and o' slots of the gradient sum to 1."""
    R = 5
    p = synth.random_params(R, seed=2).astype(np.float64)
    q = queries(4, 7, spread=1.0)
    for j in range(q.shape[0]):
        g = oracle.backward(p, q[j:j + 1], np.ones(1), R, 2)
        assert abs(g[:, 5].sum() + g[:, 9].sum() - 1.0) < 1e-13
        assert np.all(g[:, 5] >= 0) and np.all(g[:, 9] >= 0)


# ------------------------------------------------------ loss / Adam pins

def test_loss_gradients_match_torch():
    """Eq. loss (MSE) and L1 against torch's mean-reduced losses and autograd."""
    rng = synth.rng(8)
    O = rng.standard_normal(257)
    t = rng.standard_normal(257)
    t[:5] = O[:5]  # exact ties: sign(0) = 0
    for kind, fn in ((oracle.L1, torch.nn.functional.l1_loss), (oracle.MSE, torch.nn.functional.mse_loss)):
        Ot = torch.tensor(O, requires_grad=True)
        L = fn(Ot, torch.tensor(t))
        L.backward()
        gO, Lv, mae = oracle.loss_grad(O, t, kind)
        np.testing.assert_allclose(gO, Ot.grad.numpy(), rtol=1e-14, atol=1e-17)
        assert abs(Lv - L.item()) < 1e-13
        assert abs(mae - np.abs(O - t).mean()) < 1e-14


@pytest.mark.parametrize("decoupled,wd", [(False, 0.0), (False, 0.01), (True, 0.01)])
def test_adam_matches_torch_optim(decoupled, wd):
    """Adam / AdamW (Sec. 3.4, Sec. 4.2) against torch.optim in FP64, 5 steps."""
    rng = synth.rng(21)
    p0 = rng.standard_normal(103)
    pt = torch.tensor(p0.copy(), requires_grad=True)
    opt = (torch.optim.AdamW if decoupled else torch.optim.Adam)([pt], lr=1e-2, betas=(0.9, 0.999), eps=1e-8,
                                                                 weight_decay=wd)
    p, m, v = p0.copy(), np.zeros(103), np.zeros(103)
    for step in range(1, 6):
        g = rng.standard_normal(103)
        pt.grad = torch.tensor(g.copy())
        opt.step()
        p, m, v = oracle.adam(p, g, m, v, step, lr=1e-2, weight_decay=wd, decoupled=decoupled)
        np.testing.assert_allclose(p, pt.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_fit_decreases_mae_on_sphere():
    """Sec. 3.4: a few Adam iterations on the sphere SDF lower the error."""
    R = 8
    shape = synth.sphere(0.5)
    qo = synth.sample_batch(shape, 2048, seed=1).astype(np.float64)
    p = synth.init_params(R, seed=0).astype(np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    maes = []
    for step in range(1, 9):
        p, m, v, L, mae = oracle.fit_step(p, m, v, step, qo, R, loss=oracle.L1, lr=2e-2)
        maes.append(mae)
    assert all(b < a for a, b in zip(maes, maes[1:]))
    assert maes[-1] < 0.75 * maes[0]


# ------------------------------------------- backward through dO/dq pins

@pytest.mark.parametrize("R,W", [(3, 3), (6, 2)])
def test_backward_through_query_gradient_matches_central_differences(R, W):
    """The parameter gradient of L = sum gO.O + gG.dO/dq (Eq. func-normal
    differentiated once more) against FP64 central differences of the
    oracle's dO/dq, itself pinned by finite differences of O, for all 13 slots."""
    lb = oracle.default_log_beta0(R) - 1.0
    p = synth.random_params(R, seed=90 + R, delta_scale=0.6, b_scale=0.5).astype(np.float64)
    rng = synth.rng(91 + R)
    q = rng.uniform(-0.95, 0.95, (5, 3))
    if W < R:
        t = (q + 1) * R / 2 - 0.5
        frac = t - np.floor(t)
        q = np.where(np.minimum(frac, 1 - frac) < 1e-3, q + 0.01, q)
    q = q.astype(np.float32).astype(np.float64)
    gO = rng.standard_normal(q.shape[0])
    gG = rng.standard_normal((q.shape[0], 3))
    grad = oracle.backward_grad(p, q, gO, gG, R, W, lb)

    def L(pp):
        O, _, G = oracle.forward(pp, q, R, W, lb, want_dq=True)
        return float(gO @ O + (gG * G).sum())

    touched = np.flatnonzero(np.abs(grad).sum(1) > 0)
    sel = rng.choice(touched, size=min(8, touched.size), replace=False)
    an, fd = [], []
    for i in sel:
        for s in range(13):
            hstep = 1e-6 * max(1.0, abs(p[i, s]))
            pp, pm = p.copy(), p.copy()
            pp[i, s] += hstep
            pm[i, s] -= hstep
            fd.append((L(pp) - L(pm)) / (2 * hstep))
            an.append(grad[i, s])
    an, fd = np.array(an), np.array(fd)
    np.testing.assert_allclose(an, fd, rtol=2e-6, atol=2e-7 * np.abs(an).max())


def test_backward_through_query_gradient_reduces_to_plain_backward():
    """gG = 0 leaves the value term only: Algorithm 2's gradient."""
    R = 5
    p = synth.random_params(R, seed=3).astype(np.float64)
    q = queries(8, 40, spread=1.0)
    gO = synth.rng(1).standard_normal(40)
    np.testing.assert_allclose(oracle.backward_grad(p, q, gO, None, R), oracle.backward(p, q, gO, R),
                               rtol=1e-12, atol=1e-14)
    np.testing.assert_array_equal(oracle.backward_grad(p, q, None, None, R), 0.0)


def test_eikonal_loss_gradient_matches_torch():
    """Eikonal term in the squared form of Sec. 3.2, mean over queries."""
    G = synth.rng(4).standard_normal((33, 3))
    Gt = torch.tensor(G, requires_grad=True)
    Lt = 0.3 * (((Gt ** 2).sum(1) - 1.0) ** 2).mean()
    Lt.backward()
    L, gG = oracle.eikonal_loss_grad(G, weight=0.3)
    assert abs(L - Lt.item()) < 1e-14
    np.testing.assert_allclose(gG, Gt.grad.numpy(), rtol=1e-13, atol=1e-15)


# -------------------------------------------------- mean-shift init pins

def test_mean_shift_single_point_and_symmetric_pair():
    """Sec. 3.3: with one surface point every centre's offset points at it;
    with two points equidistant from a centre the offset points at their
    midpoint."""
    R = 4
    k = centres(R)
    s = np.array([[0.3, -0.2, 0.1]])
    np.testing.assert_allclose(oracle.mean_shift(s, R), s - k, rtol=0, atol=1e-15)
    # two points mirrored through centre 0
    d = np.array([0.1, 0.05, -0.2])
    pts = np.stack([k[0] + d, k[0] - d])
    np.testing.assert_allclose(oracle.mean_shift(pts, R)[0], 0.0, atol=1e-15)


def test_mean_shift_bandwidth_limits():
    """Large bandwidth: the weight concentrates on the nearest point (argmin
    of the distance); small bandwidth: all points weigh the same (the mean)."""
    R = 3
    pts = synth.rng(5).uniform(-1, 1, (50, 3))
    k = centres(R)
    near = pts[np.argmin(scipy.spatial.distance.cdist(k, pts, "sqeuclidean"), axis=1)]
    np.testing.assert_allclose(oracle.mean_shift(pts, R, bandwidth=1e6), near - k, atol=1e-9)
    np.testing.assert_allclose(oracle.mean_shift(pts, R, bandwidth=1e-9), pts.mean(0) - k, atol=1e-8)


def test_mean_shift_far_centres_stay_defined():
    """Points far from a centre (every exp(-100 d^2) underflows in FP64) still
    give a finite offset, equal to the large-bandwidth (nearest point) limit
    when one point dominates."""
    pts = np.array([[0.9, 0.9, 0.9], [0.95, 0.9, 0.9]])
    d = oracle.mean_shift(pts, 2, bandwidth=1000.0)
    assert np.all(np.isfinite(d))
    k = centres(2)
    np.testing.assert_allclose(d[0], pts[0] - k[0], atol=1e-12)


# ------------------------------------------------ ablation variant pins

def taylor_params(R, sets, deg, learn, seed, global_poly):
    """Parameters of a variant whose every key holds the Taylor coefficients,
    about its own position, of one global polynomial P of degree <= deg
    (P(x) = c + g.x + 1/2 x^T H x + 1/6 T[x,x,x], H and T symmetric)."""
    c, gv, H, T = global_poly
    ch = oracle.variant_channels(sets, deg, learn)
    rng = synth.rng(seed)
    p = np.zeros((R ** 3, ch))
    k = centres(R)
    base = 0
    if sets & 2:
        p[:, 0:3] = rng.uniform(-0.4, 0.4, (R ** 3, 3)) * (2.0 / R)
        base = 3
    nsets = (sets & 1) + ((sets >> 1) & 1)
    if learn:
        p[:, base:base + nsets] = rng.normal(0.0, 0.5, (R ** 3, nsets))
    nv = [1, 4, 10, 20][deg]
    off = base + learn * nsets
    tri = [(0, 0, 0), (1, 1, 1), (2, 2, 2), (0, 0, 1), (0, 0, 2), (0, 1, 1), (1, 1, 2), (0, 2, 2), (1, 2, 2), (0, 1, 2)]
    for s_i, s in enumerate([s for s in (0, 1) if sets & (1 << s)]):
        pos = k + (p[:, 0:3] if s == 1 else 0.0)
        val = c + pos @ gv + 0.5 * np.einsum("na,ab,nb->n", pos, H, pos) + np.einsum("abc,na,nb,nc->n", T, pos, pos, pos) / 6
        grad = gv + pos @ H + 0.5 * np.einsum("abc,nb,nc->na", T, pos, pos)
        hess = H + np.einsum("abc,nc->nab", T, pos)
        phi = np.zeros((R ** 3, 20))
        phi[:, 0] = val
        phi[:, 1:4] = grad
        phi[:, 4:7] = hess[:, [0, 1, 2], [0, 1, 2]]
        phi[:, 7] = hess[:, 0, 1]
        phi[:, 8] = hess[:, 0, 2]
        phi[:, 9] = hess[:, 1, 2]
        for i, (a, b, cc) in enumerate(tri):
            phi[:, 10 + i] = T[a, b, cc]
        p[:, off + s_i * nv: off + (s_i + 1) * nv] = phi[:, :nv]
    return p


def random_global_poly(deg, seed):
    rng = synth.rng(seed)
    c = rng.normal()
    g = rng.normal(size=3) if deg >= 1 else np.zeros(3)
    H = rng.normal(size=(3, 3)) if deg >= 2 else np.zeros((3, 3))
    H = H + H.T
    T = np.zeros((3, 3, 3))
    if deg >= 3:
        A = rng.normal(size=(3, 3, 3))
        import itertools
        for perm in itertools.permutations(range(3)):
            T += np.transpose(A, perm)
        T /= 6
    return c, g, H, T


def test_variant_channels_match_table_ablation():
    """Column 'Ch' and '# Params' of Table tab:ablation for every grid and
    full configuration: the oracle's channel count for (sets, deg, learn)."""
    g = json.load(open(os.path.join(GOLDEN, "param_counts.json")))
    for r in g["table_ablation"]:
        ch = oracle.variant_channels(*r["variant"])
        assert ch == r["floats_per_centre"], r["config"]
        assert r["R"] ** 3 * ch == r["value"], r["config"]
    assert oracle.variant_channels(0, 1, 1) == -1 and oracle.variant_channels(1, 4, 1) == -1


@pytest.mark.parametrize("R,W", [(3, 3), (6, 2)])
def test_variant_default_layout_reduces_to_the_pinned_model(R, W):
    """sets = 3, deg = 1, learn = 1 is the 13-float model of Eq. func-offset:
    forward and backward equal the oracle's (pinned) main functions."""
    p = synth.random_params(R, seed=31 + R, delta_scale=0.6, b_scale=0.5).astype(np.float64)
    q = queries(32 + R, 60)
    O, lse = oracle.variant_forward(p, q, R, 3, 1, 1, W)
    O0, lse0 = oracle.forward(p, q, R, W)[:2]
    np.testing.assert_allclose(O, O0, rtol=0, atol=1e-14)
    np.testing.assert_allclose(lse, lse0, rtol=0, atol=1e-12)
    gO = synth.rng(33).standard_normal(q.shape[0])
    np.testing.assert_allclose(oracle.variant_backward(p, q, gO, R, 3, 1, 1, W), oracle.backward(p, q, gO, R, W),
                               rtol=0, atol=1e-13)


@pytest.mark.parametrize("sets", [1, 2, 3])
@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_variant_polynomial_reproduction(sets, deg):
    """Eq. poly-func in Taylor form is exact for polynomials of its degree:
    when every key holds the Taylor coefficients of one global polynomial P
    (deg <= the value degree) about its own position, the softmax blend is
    P(q) for any scales and offsets (partition of unity + shift invariance).
    A wrong 1/2 or 1/6 factor, a wrong symmetric multiplicity or a swapped
    coefficient breaks it."""
    R = 4
    for learn in (0, 1):
        P = random_global_poly(deg, 40 + 4 * deg + sets)
        p = taylor_params(R, sets, deg, learn, 50 + sets, P)
        q = queries(60 + deg, 80, spread=1.05)
        O, _ = oracle.variant_forward(p, q, R, sets, deg, learn)
        c, g, H, T = P
        exact = c + q @ g + 0.5 * np.einsum("na,ab,nb->n", q, H, q) + np.einsum("abc,na,nb,nc->n", T, q, q, q) / 6
        np.testing.assert_allclose(O, exact, rtol=0, atol=1e-11 * max(1.0, np.abs(exact).max()))
        # every key agrees with the blend, so the log-scale gradients vanish
        if learn:
            gO = synth.rng(7).standard_normal(q.shape[0])
            grad = oracle.variant_backward(p, q, gO, R, sets, deg, learn)
            b0 = 3 if sets & 2 else 0
            nsets = (sets & 1) + ((sets >> 1) & 1)
            np.testing.assert_allclose(grad[:, b0:b0 + nsets], 0.0, atol=1e-10)


def test_variant_degree0_fixed_scale_is_the_normalised_rbf():
    """Config-G-1 (grid keys, degree 0, fixed scale) is Eq. nrbf: the blend
    of the values with scipy's softmax of -beta |q - k|^2 over the window."""
    R, W = 3, 3
    lb = 2.0
    v = synth.rng(5).standard_normal(R ** 3)
    q = queries(6, 50)
    O, _ = oracle.variant_forward(v[:, None], q, R, 1, 0, 0, W, lb)
    d2 = scipy.spatial.distance.cdist(q, centres(R), "sqeuclidean")
    ref = (scipy.special.softmax(-math.exp(lb) * d2, axis=1) * v[None, :]).sum(1)
    np.testing.assert_allclose(O, ref, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("sets,deg,learn", [(1, 0, 0), (1, 1, 1), (1, 2, 1), (1, 3, 0), (2, 1, 1), (2, 3, 1),
                                            (3, 2, 1)])
def test_variant_gradients_match_central_differences(sets, deg, learn):
    """The variant backward (Algorithm 2 closed forms with the polynomial's
    own gradient for the key offset) against FP64 central differences of the
    variant forward, every channel of a sample of touched centres."""
    R = 4
    ch = oracle.variant_channels(sets, deg, learn)
    rng = synth.rng(70 + deg + 4 * sets)
    p = rng.normal(0.0, 0.3, (R ** 3, ch))
    if sets & 2:
        p[:, 0:3] = rng.uniform(-0.3, 0.3, (R ** 3, 3)) * (2.0 / R)
    lb = oracle.default_log_beta0(R) - 1.0
    q = rng.uniform(-0.9, 0.9, (6, 3))
    t = (q + 1) * R / 2 - 0.5
    frac = t - np.floor(t)
    q = np.where(np.minimum(frac, 1 - frac) < 1e-3, q + 0.01, q).astype(np.float32).astype(np.float64)
    gO = rng.standard_normal(q.shape[0])
    grad = oracle.variant_backward(p, q, gO, R, sets, deg, learn, 2, lb)

    def L(pp):
        return float(gO @ oracle.variant_forward(pp, q, R, sets, deg, learn, 2, lb)[0])

    touched = np.flatnonzero(np.abs(grad).sum(1) > 0)
    sel = rng.choice(touched, size=min(6, touched.size), replace=False)
    an, fd = [], []
    for i in sel:
        for s in range(ch):
            hstep = 1e-6 * max(1.0, abs(p[i, s]))
            pp, pm = p.copy(), p.copy()
            pp[i, s] += hstep
            pm[i, s] -= hstep
            fd.append((L(pp) - L(pm)) / (2 * hstep))
            an.append(grad[i, s])
    an, fd = np.array(an), np.array(fd)
    np.testing.assert_allclose(an, fd, rtol=2e-6, atol=2e-8 * max(1.0, np.abs(an).max()))


# ------------------------------------------- cosine-series decomposition pins

def test_cosine_series_one_band_is_config_g6():
    """Sec. 4.4: with one band (b = 0, weight cos 0 = 1) the decomposition is
    Config-G-6 at the same resolution."""
    R = 5
    p = synth.variant_params(synth.random_union(3), R, 1, 1, 1, seed=3).astype(np.float64)
    q = queries(4, 70)
    S = oracle.cosine_forward(p[None], q, R, 1)
    O, _ = oracle.variant_forward(p, q, R, 1, 1, 1)
    np.testing.assert_allclose(S, O, rtol=0, atol=1e-15)
    gS = synth.rng(5).standard_normal(q.shape[0])
    np.testing.assert_allclose(oracle.cosine_backward(p[None], q, gS, R, 1)[0],
                               oracle.variant_backward(p, q, gS, R, 1, 1, 1), rtol=0, atol=1e-14)


def test_cosine_series_of_constant_bands_is_the_cosine_sum():
    """Bands holding constant values c_b (partition of unity: O_b = c_b for
    any scales) give S(q) = sum_b c_b cos(b pi x) cos(b pi y) cos(b pi z),
    the truncated Fourier cosine series of Eq. cosine-series."""
    R, B = 4, 5
    rng = synth.rng(8)
    c = rng.standard_normal(B)
    p = np.zeros((B, R ** 3, 5))
    p[:, :, 0] = rng.normal(0.0, 0.5, (B, R ** 3))
    p[:, :, 1] = c[:, None]
    q = queries(9, 100, spread=1.0)
    S = oracle.cosine_forward(p, q, R, B)
    b = np.arange(B)[None, :]
    ref = (c[None, :] * np.cos(b * np.pi * q[:, 0:1]) * np.cos(b * np.pi * q[:, 1:2]) *
           np.cos(b * np.pi * q[:, 2:3])).sum(1)
    np.testing.assert_allclose(S, ref, rtol=0, atol=1e-13)


def test_cosine_series_gradients_match_central_differences():
    R, B = 4, 3
    rng = synth.rng(12)
    p = rng.normal(0.0, 0.3, (B, R ** 3, 5))
    lb = oracle.default_log_beta0(R) - 1.0
    q = rng.uniform(-0.9, 0.9, (5, 3))
    t = (q + 1) * R / 2 - 0.5
    frac = t - np.floor(t)
    q = np.where(np.minimum(frac, 1 - frac) < 1e-3, q + 0.01, q).astype(np.float32).astype(np.float64)
    gS = rng.standard_normal(q.shape[0])
    grad = oracle.cosine_backward(p, q, gS, R, B, 2, lb)
    flat = grad.reshape(-1, 5)
    touched = np.flatnonzero(np.abs(flat).sum(1) > 0)
    sel = rng.choice(touched, size=min(8, touched.size), replace=False)
    an, fd = [], []
    for i in sel:
        for s in range(5):
            hstep = 1e-6 * max(1.0, abs(p.reshape(-1, 5)[i, s]))
            pp, pm = p.copy().reshape(-1, 5), p.copy().reshape(-1, 5)
            pp[i, s] += hstep
            pm[i, s] -= hstep
            fd.append((gS @ oracle.cosine_forward(pp, q, R, B, 2, lb) - gS @ oracle.cosine_forward(pm, q, R, B, 2, lb))
                      / (2 * hstep))
            an.append(flat[i, s])
    np.testing.assert_allclose(np.array(an), np.array(fd), rtol=2e-6, atol=2e-8 * max(1.0, np.abs(an).max()))


# ------------------------------------------------- tolerance diagnostics

def test_kappa_is_the_attained_first_order_sensitivity():
    """kappa, from which the FP32 forward tolerance is derived, is the first
    order worst case of O under relative perturbations of size eps of every
    key's exponent and weight: the adversarial perturbation (exponent by
    eps sign((f - O) expo), weight by eps sign(f - O)) moves O by eps kappa,
    and random perturbations of the same size by less."""
    R, lb, eps = 3, 2.0, 1e-7
    p = synth.random_params(R, seed=77, delta_scale=0.6, b_scale=0.6).astype(np.float64)
    q = queries(78, 16)
    O, _, kappa = oracle.forward(p, q, R, W=R, log_beta0=lb, want_kappa=True)
    pos, beta, o, d = keys_of(p, R, lb)
    rng = synth.rng(79)

    def blend(ex, w, f):
        lw = np.exp(ex - ex.max()) * w
        return (lw * f).sum() / lw.sum()

    for j in range(q.shape[0]):
        r = q[j] - pos
        expo = -beta * (r ** 2).sum(1)
        f = o + (d * r).sum(1)
        s = np.sign(f - O[j])
        worst = blend(expo * (1 + eps * s * np.sign(expo)), 1 + eps * s, f)
        assert abs(abs(worst - O[j]) / eps - kappa[j]) <= 1e-5 * kappa[j] + 1e-8
        for _ in range(3):
            rnd = blend(expo * (1 + eps * rng.uniform(-1, 1, expo.size)), 1 + eps * rng.uniform(-1, 1, expo.size), f)
            assert abs(rnd - O[j]) <= eps * kappa[j] * (1 + 1e-5) + 1e-15


def _G_direct(expo, w, g):
    """G = sum softmax g over keys with exponents expo and extra weights w,
    each key's term g (n, 3) held fixed: the direct dependence of dO/dq on
    the weights (O, inside g, not recomputed)."""
    lw = np.exp(expo - expo.max()) * w
    return (lw[:, None] * g).sum(0) / lw.sum()


def test_dq_error_terms_are_attained_and_bound_random_perturbations():
    """The error terms from which the FP32 tolerance of dO/dq is derived.
    kappa_G bounds the first-order change of G = dO/dq (Eq. func-normal)
    under relative perturbations eps of every exponent and weight with O held
    fixed; with two keys (R = 1) the terms g_i - G are collinear and the
    adversarial perturbation along them attains eps kappa_G.  fabs is
    attained by perturbing every term of every value f by eps in the sign of
    the term (O moves by eps fabs), gabs likewise by the terms of G along
    each axis (G_a moves by at most eps gabs), and random perturbations stay
    below both."""
    eps = 1e-7
    for R, lb, seed in ((1, 1.5, 91), (3, 2.0, 92)):
        p = synth.random_params(R, seed=seed, delta_scale=0.6, b_scale=0.6).astype(np.float64)
        q = queries(seed + 1, 12)
        O, _, G = oracle.forward(p, q, R, W=R, log_beta0=lb, want_dq=True)
        kG, fab, gab = oracle.dq_error_terms(p, q, R, W=R, log_beta0=lb)
        pos, beta, o, d = keys_of(p, R, lb)
        rng = synth.rng(seed + 2)
        for j in range(q.shape[0]):
            r = q[j] - pos
            expo = -beta * (r ** 2).sum(1)
            f = o + (d * r).sum(1)
            sm = np.exp(expo - expo.max())
            sm /= sm.sum()
            g = d + 2.0 * beta[:, None] * r * (O[j] - f)[:, None]
            assert np.allclose(_G_direct(expo, np.ones_like(expo), g), G[j], rtol=1e-12, atol=1e-12)
            if R == 1:
                e = g[0] - g[1]
                e = e / np.linalg.norm(e)
                s = np.sign((g - G[j]) @ e)
                worst = _G_direct(expo * (1 + eps * s * np.sign(expo)), 1 + eps * s, g)
                assert abs(abs((worst - G[j]) @ e) / eps - kG[j]) <= 1e-5 * kG[j] + 1e-8
            for _ in range(3):
                rnd = _G_direct(expo * (1 + eps * rng.uniform(-1, 1, expo.size)),
                                1 + eps * rng.uniform(-1, 1, expo.size), g)
                assert np.linalg.norm(rnd - G[j]) <= eps * kG[j] * (1 + 1e-5) + 1e-15
            # fabs: every term of f perturbed by eps in its own sign
            terms = np.concatenate([o[:, None], d * r], 1)
            f_up = (terms * (1 + eps * np.sign(terms))).sum(1)
            assert abs(((sm * f_up).sum() - O[j]) / eps - fab[j]) <= 1e-5 * fab[j] + 1e-8
            f_rnd = (terms * (1 + eps * rng.uniform(-1, 1, terms.shape))).sum(1)
            assert abs((sm * f_rnd).sum() - O[j]) <= eps * fab[j] * (1 + 1e-5) + 1e-15
            # gabs: the terms d_a and 2 beta r_a (O - f) of G_a perturbed likewise
            ta = np.stack([d, 2.0 * beta[:, None] * r * (O[j] - f)[:, None]], 2)   # (keys, axis, term)
            moved = (sm[:, None] * (ta * eps * np.sign(ta)).sum(2)).sum(0)
            assert np.linalg.norm(moved) <= eps * gab[j] * (1 + 1e-9) + 1e-15
            assert np.linalg.norm(moved) >= eps * gab[j] / np.sqrt(3) * (1 - 1e-9) - 1e-15


def test_backward_error_terms_bound_the_gradient_and_are_attained_by_one_query():
    """abs0, the magnitudes of every gradient entry's terms, bounds |grad|
    entry by entry (triangle inequality) and equals it where a single query
    contributes terms of one sign (its o and o' entries: dL/dO times a
    weight); abs1 weighs each term by (|exponent| + 1) >= 1 of its key."""
    R, lb = 3, 2.0
    p = synth.random_params(R, seed=93, delta_scale=0.6, b_scale=0.6).astype(np.float64)
    q = queries(94, 40)
    gO = synth.rng(95).standard_normal(q.shape[0])
    g = oracle.backward(p, q, gO, R, W=R, log_beta0=lb)
    a0, a1 = oracle.backward_error_terms(p, q, gO, R, W=R, log_beta0=lb)
    assert np.all(np.abs(g) <= a0 * (1 + 1e-12) + 1e-300)
    assert np.all(a1 >= a0 * (1 - 1e-12))
    for j in range(3):
        gj = oracle.backward(p, q[j:j + 1], gO[j:j + 1], R, W=R, log_beta0=lb)
        b0, b1 = oracle.backward_error_terms(p, q[j:j + 1], gO[j:j + 1], R, W=R, log_beta0=lb)
        for slot in (5, 9):
            np.testing.assert_allclose(b0[:, slot], np.abs(gj[:, slot]), rtol=1e-12, atol=1e-300)
        # the (|exponent| + 1) weight of one query's o entries: the key's own exponent
        O, lse = oracle.forward(p, q[j:j + 1], R, W=R, log_beta0=lb)
        pos, beta, o, d = keys_of(p, R, lb)
        expo = -beta * ((q[j] - pos) ** 2).sum(1)
        ng = R ** 3
        np.testing.assert_allclose(b1[:, 5], b0[:, 5] * (np.abs(expo[:ng]) + 1), rtol=1e-12, atol=1e-300)
        # the Delta entries: |-d + 2 beta (q - p)(f - O)| equals its bound
        # |d| + 2 beta |q - p| |f - O| where the two parts share a sign
        r = q[j] - pos[ng:]
        f = o[ng:] + (d[ng:] * r).sum(1)
        part1 = -d[ng:]
        part2 = 2.0 * beta[ng:, None] * r * (f - O[0])[:, None]
        same = np.sign(part1) == np.sign(part2)
        assert same.any() and (~same).any()
        np.testing.assert_allclose(b0[:, 0:3][same], np.abs(gj[:, 0:3][same]), rtol=1e-10, atol=1e-300)
        assert np.all(b0[:, 0:3][~same] > np.abs(gj[:, 0:3][~same]))


def test_dq_sensitivity_is_the_norm_of_the_lse_gradient():
    """dq_sens = 2 ||sum softmax beta (q - key)||, the factor by which an
    error in O enters dO/dq, equals ||grad_q lse|| (lse = log sum
    exp(-beta ||q - key||^2)): central differences of the oracle's lse."""
    R, lb, h = 3, 2.0, 1e-6
    p = synth.random_params(R, seed=81, delta_scale=0.6, b_scale=0.6).astype(np.float64)
    q = queries(82, 12)
    _, _, sens = oracle.forward(p, q, R, W=R, log_beta0=lb, want_dq_sens=True)
    grad = np.zeros((q.shape[0], 3))
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        _, lp = oracle.forward(p, q + e, R, W=R, log_beta0=lb)
        _, lm = oracle.forward(p, q - e, R, W=R, log_beta0=lb)
        grad[:, a] = (lp - lm) / (2 * h)
    np.testing.assert_allclose(sens, np.linalg.norm(grad, axis=1), rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_variant_fabs_of_a_single_key_is_the_sum_of_its_taylor_terms(deg):
    """fabs, from which the variant tolerance is derived, is for a single key
    (R = 1, grid keys only: softmax 1) the sum of the absolute values of the
    distinct Taylor terms of f at x = q - key: |o|, |d_a x_a|, |S_aa x_a^2| / 2,
    |S_ab x_a x_b| (a < b), |T_aaa x_a^3| / 6, |T_aab x_a^2 x_b| / 2 (a != b),
    |T_xyz x y z|, with the channel order of Eq. func-offset's tuple."""
    rng = synth.rng(90 + deg)
    nv = [1, 4, 10, 20][deg]
    for _ in range(5):
        phi = rng.uniform(-2, 2, nv)
        p = np.concatenate([[rng.uniform(-1, 1)], phi])[None, :]   # (b, phi)
        x = rng.uniform(-0.8, 0.8, (4, 3))
        _, _, kap, fab = oracle.variant_forward(p, x, 1, 1, deg, 1, log_beta0=1.0, want_diag=True)
        for j in range(4):
            X, Y, Z = x[j]
            terms = [phi[0]]
            if deg >= 1:
                terms += [phi[1] * X, phi[2] * Y, phi[3] * Z]
            if deg >= 2:
                terms += [phi[4] * X * X / 2, phi[5] * Y * Y / 2, phi[6] * Z * Z / 2,
                          phi[7] * X * Y, phi[8] * X * Z, phi[9] * Y * Z]
            if deg >= 3:
                terms += [phi[10] * X ** 3 / 6, phi[11] * Y ** 3 / 6, phi[12] * Z ** 3 / 6,
                          phi[13] * X * X * Y / 2, phi[14] * X * X * Z / 2, phi[15] * X * Y * Y / 2,
                          phi[16] * Y * Y * Z / 2, phi[17] * X * Z * Z / 2, phi[18] * Y * Z * Z / 2,
                          phi[19] * X * Y * Z]
            assert abs(fab[j] - np.abs(terms).sum()) <= 1e-12 * (1 + np.abs(terms).sum())
            assert abs(kap[j]) <= 1e-12   # one key: f - O = 0
