"""GPU parity of the mean-shift offset initialisation (Sec. 3.3) against the
FP64 oracle, on surface points of seeded synthetic shapes.

Error model (FP32 kernel, base-2 exponent, FP64 oracle).  The kernel scales
coordinates by sigma = sqrt(bw log2(e)), so the base-2 exponent of a pair is
e_n = -|sigma s_n - sigma k_i|^2.  For centre i with largest exponent M_i:
  * each scaled difference is off by at most u sigma (|s| + |k| + |r|)
    <= 4 u sigma per component, which moves e_n by at most
    8 sqrt(3) u sigma |r| = 14 u sigma sqrt(|e_n|); the squares and sums add
    3u |e_n|.  The kernel subtracts a reference M within 64 of M_i, with one
    more rounding, so the ratio of two contributing weights
    (e_n - M_i > -40) is off by a factor 2^delta with
    |delta| <= u (6 (|M_i| + 40) + 28 sigma sqrt(|M_i| + 40) + 300)
    (300 covers the subtraction of at most 104 and ex2);
  * the weighted sums are accumulated sequentially by 32 lanes of N/256
    points each (8 CTAs of a cluster split the points), with at most as many
    rescales, and merged in 8 steps: relative error at most (N/2 + 16) u of
    sum w |r| (a generous bound);
  * the offset is S/Z with S = sum w (s - k), so both effects enter scaled by
    rho_i + |Delta_i|, rho_i = max |s_n - k_i| over contributing points; the
    scaled differences and the final division by Z sigma add 8u;
  * points below 2^-40 of the largest weight add at most N 2^-40 max|r|.
This gives a worst-case bound per centre; the typical error is far smaller
and is asserted separately in the random-rounding model (sqrt(N/8) u).
R = 5 leaves 3 of the 4 centre slots of every second warp empty (ragged c);
N < 8 leaves some CTAs of a cluster without points."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2505_21319_gb300 import api, synth

pytestmark = pytest.mark.gpu

DEV = "cuda"
U = 2.0 ** -24
LOG2E = 1.4426950408889634


def centres(R):
    c = -1.0 + (np.arange(R) + 0.5) * (2.0 / R)
    a, b, d = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([a.ravel(), b.ravel(), d.ravel()], 1)


def error_bound(pts, R, bw, delta, idx):
    """Worst-case |gpu - oracle| per centre idx (module docstring)."""
    k = centres(R)[idx]
    sigma = math.sqrt(bw * LOG2E)
    s = pts.astype(np.float64)
    N = s.shape[0]
    out = np.empty(len(idx))
    for a in range(0, len(idx), 128):
        kk = k[a:a + 128]
        r = s[None, :, :] - kk[:, None, :]
        e = -bw * LOG2E * np.einsum("cnk,cnk->cn", r, r)
        M = e.max(1)
        contrib = e - M[:, None] > -40
        rn = np.sqrt(np.einsum("cnk,cnk->cn", r, r))
        rho = np.where(contrib, rn, 0).max(1)
        dnorm = np.abs(delta[idx[a:a + 128]]).max(1)
        Mc = np.abs(M) + 40
        delta_w = math.log(2) * (6 * Mc + 28 * sigma * np.sqrt(Mc) + 300)
        out[a:a + 128] = U * (delta_w + N / 2 + 16) * (rho + dnorm) + 8 * U + N * 2.0 ** -40 * 3.5 + 1e-7
    return out


def run_gpu(pts, R, bw=100.0, params=None):
    if params is None:
        params = torch.zeros(R ** 3 * 13, dtype=torch.float32, device=DEV)
    api.efunc_mean_shift_init(params, torch.from_numpy(np.ascontiguousarray(pts, np.float32)).to(DEV), bw)
    torch.cuda.synchronize()
    return params.cpu().numpy().reshape(-1, 13)


def shape_points(seed, N):
    return synth.surface_points(synth.random_union(seed), N, synth.rng(seed)).astype(np.float32)


def check(pts, R, bw=100.0, idx=None, typical=True):
    ref = oracle.mean_shift(pts, R, bw)
    got = run_gpu(pts, R, bw)[:, :3].astype(np.float64)
    idx = np.arange(R ** 3) if idx is None else idx
    err = np.abs(got[idx] - ref[idx]).max(1)
    lim = error_bound(pts, R, bw, ref, idx)
    bad = np.flatnonzero(~(err <= lim))
    assert bad.size == 0, (f"R={R} N={len(pts)}: {bad.size} centres outside the bound; worst "
                           f"{idx[bad[:4]]} err {err[bad[:4]]} lim {lim[bad[:4]]}")
    # random-rounding model: typical error ~ sqrt(N/8) u (rho + |Delta|), rho+|Delta| <= 2 sqrt(3)
    if typical:
        lim_t = math.sqrt(len(pts) / 8 + 64) * U * 2 * math.sqrt(3) * 8
        assert np.median(err) <= lim_t, (np.median(err), lim_t)
    return err


@pytest.mark.parametrize("R,N,seed", [(4, 100, 1), (5, 1025, 2), (8, 3000, 3), (8, 7, 6), (16, 16384, 4), (8, 40000, 8)])
def test_mean_shift_matches_oracle(R, N, seed):
    """Ragged centre groups (R=5), ragged point shares (1025, 3000), fewer
    points than CTAs per cluster (7), the paper's N = 16384 surface points,
    and more points than one tile per CTA (40000)."""
    check(shape_points(seed, N), R)


def test_mean_shift_full_size_sampled():
    """R = 32, N = 16384 (the paper's setting): every centre against the
    oracle's exact value, the bound evaluated on a sample of 2048 centres
    (all eight corners included) and a loose bound everywhere."""
    R, N = 32, 16384
    pts = shape_points(7, N)
    ref = oracle.mean_shift(pts, R)
    got = run_gpu(pts, R)[:, :3].astype(np.float64)
    err = np.abs(got - ref).max(1)
    g = synth.rng(7)
    corners = np.array([((a * R + b) * R + c) for a in (0, R - 1) for b in (0, R - 1) for c in (0, R - 1)])
    idx = np.unique(np.concatenate([corners, g.integers(0, R ** 3, 2048)]))
    lim = error_bound(pts, R, 100.0, ref, idx)
    assert np.all(err[idx] <= lim), (err[idx].max(), lim.min())
    # the worst-case bound never exceeds its value at |M| = 1731 (|k - s|^2 <= 12), rho + |Delta| <= 2 sqrt(12)
    Mc, sigma = 1731 + 40, math.sqrt(100 * LOG2E)
    assert err.max() <= U * (math.log(2) * (6 * Mc + 28 * sigma * math.sqrt(Mc) + 300) + N / 2 + 16) * 2 * math.sqrt(12)
    assert np.median(err) <= 1e-5


def test_mean_shift_single_point_is_the_difference():
    """N = 1: every weight is 1, so Delta_i = s - k_i (one FP32 rounding)."""
    R = 8
    s = np.array([[0.3, -0.7, 0.11]], np.float32)
    got = run_gpu(s, R)[:, :3].astype(np.float64)
    ref = s.astype(np.float64) - centres(R)
    assert np.all(np.abs(got - ref) <= U * np.abs(ref) + 1e-7)


def test_mean_shift_leaves_other_slots_untouched():
    R = 8
    p = torch.from_numpy(synth.random_params(R, 11)).to(DEV).reshape(-1).contiguous()
    before = p.cpu().numpy().reshape(-1, 13).copy()
    pts = shape_points(11, 2000)
    after = run_gpu(pts, R, params=p)
    assert np.array_equal(after[:, 3:], before[:, 3:])
    ref = oracle.mean_shift(pts, R)
    assert np.all(np.abs(after[:, :3] - ref).max(1) <= error_bound(pts, R, 100.0, ref, np.arange(R ** 3)))


@pytest.mark.parametrize("bw", [1.0, 1e4])
def test_mean_shift_bandwidths(bw):
    """A wide kernel (bw = 1: nearly the mean of all points) and a narrow one
    (bw = 1e4: nearly the nearest point, exponents down to -1.7e5 whose
    shift must not underflow)."""
    check(shape_points(5, 4000), 8, bw, typical=bw == 1.0)


def test_mean_shift_moves_offset_keys_onto_the_surface():
    """With the offsets initialised, the offset keys of centres within one
    cell of the surface sit much closer to it: the median |SDF(k_i + Delta_i)|
    drops below 0.4 of the median |SDF(k_i)| (the oracle gives 0.24 on this
    shape; curvature keeps it from reaching 0)."""
    R = 16
    shape = synth.random_union(9)
    pts = synth.surface_points(shape, 16384, synth.rng(9)).astype(np.float32)
    got = run_gpu(pts, R)[:, :3].astype(np.float64)
    moved = centres(R) + got
    near = np.abs(shape.sdf(centres(R))) < 2.0 / R
    assert np.median(np.abs(shape.sdf(moved[near]))) < 0.4 * np.median(np.abs(shape.sdf(centres(R)[near])))
