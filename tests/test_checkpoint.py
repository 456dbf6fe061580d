"""Checkpoint / resume (host code, CPU): the file round-trips the arrays bit
for bit with the fit's configuration, every kind of damage is reported as
EFUNC_ERR_IO rather than loaded, and a fit resumed from a checkpoint follows
the uninterrupted oracle trajectory exactly."""
import ctypes
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2505_21319_gb300 import _binding as B
from paper_2505_21319_gb300 import api, synth


def _state(n, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.randn(n, generator=g), torch.randn(n, generator=g), torch.rand(n, generator=g)


@pytest.mark.parametrize("R,channels", [(8, 13), (4, 5), (16, 10), (1, 21)])
def test_round_trip_is_bit_exact(tmp_path, R, channels):
    n = R ** 3 * channels
    p, m, v = _state(n, R + channels)
    path = tmp_path / "fit.ckp"
    api.save_checkpoint(path, p, m, v, step=123, channels=channels, seed=99, loss="mse", lr=6e-4,
                        weight_decay=0.01, decoupled=True, log_beta0=3.5)
    c = api.load_checkpoint(path, device="cpu")
    for name, t in (("params", p), ("m", m), ("v", v)):
        assert torch.equal(c[name], t), name
    assert (c["step"], c["seed"], c["loss"], c["R"], c["W"], c["channels"]) == (123, 99, "mse", R, 2, channels)
    assert c["log_beta0"] == 3.5
    assert c["adam"] == {"lr": 6e-4, "beta1": 0.9, "beta2": 0.999, "eps": 1e-8, "weight_decay": 0.01,
                         "decoupled": True}
    assert os.path.getsize(path) == 128 + 12 * n + 8
    assert sorted(os.listdir(tmp_path)) == ["fit.ckp"]   # no temporary file left behind


def _damaged(tmp_path, edit):
    p, m, v = _state(4 ** 3 * 13, 1)
    path = tmp_path / "d.ckp"
    api.save_checkpoint(path, p, m, v, step=3)
    data = bytearray(path.read_bytes())
    path.write_bytes(bytes(edit(data)))
    with pytest.raises(B.EfuncError) as info:
        api.load_checkpoint(path, device="cpu")
    return info.value.code


def _flip(pos):
    def edit(d):
        d[pos] ^= 0x10
        return d
    return edit


@pytest.mark.parametrize("what,edit", [
    ("magic", _flip(0)),
    ("version", _flip(8)),
    ("a header field", _flip(40)),
    ("the header checksum", _flip(121)),
    ("a parameter", _flip(128 + 4 * 100 + 2)),
    ("a second moment", _flip(128 + 2 * 4 * 832 + 7)),
    ("the payload checksum", lambda d: _flip(len(d) - 3)(d)),
    ("one byte short", lambda d: d[:-1]),
    ("one byte more", lambda d: d + b"\0"),
    ("header only", lambda d: d[:128]),
    ("empty", lambda d: bytearray()),
])
def test_damage_is_reported_not_loaded(tmp_path, what, edit):
    assert _damaged(tmp_path, edit) == 6, what


def test_argument_and_file_errors(tmp_path):
    lib = B.load()
    with pytest.raises(B.EfuncError) as info:
        api.load_checkpoint(tmp_path / "missing.ckp", device="cpu")
    assert info.value.code == 6
    n = 2 ** 3 * 13
    p, m, v = (np.zeros(n, np.float32) for _ in range(3))
    good = B.CheckpointInfo(2, 2, 7.0, 13, n, 0, 0, 0, api.make_adam())
    ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    path = str(tmp_path / "x.ckp").encode()
    assert lib.efunc_checkpoint_save(path, ctypes.byref(good), ptr(p), ptr(m), ptr(v)) == 0
    for field, value in (("n", n + 1), ("step", -1), ("channels", 0), ("R", 0), ("W", 0)):
        bad = B.CheckpointInfo(2, 2, 7.0, 13, n, 0, 0, 0, api.make_adam())
        setattr(bad, field, value)
        assert lib.efunc_checkpoint_save(path, ctypes.byref(bad), ptr(p), ptr(m), ptr(v)) == 1, field
    assert lib.efunc_checkpoint_save(path, ctypes.byref(good), None, ptr(m), ptr(v)) == 1
    assert lib.efunc_checkpoint_save(str(tmp_path / "no" / "dir.ckp").encode(), ctypes.byref(good), ptr(p), ptr(m),
                                     ptr(v)) == 6
    info = B.CheckpointInfo()
    assert lib.efunc_checkpoint_load(path, ctypes.byref(info), ptr(p), ptr(m), ptr(v), n - 1) == 1   # too small
    assert lib.efunc_checkpoint_load(path, ctypes.byref(info), ptr(p), ptr(m), ptr(v), n) == 0
    assert lib.efunc_checkpoint_info_read(path, None) == 1
    with pytest.raises(ValueError):
        api.save_checkpoint(tmp_path / "y.ckp", torch.zeros(100), torch.zeros(100), torch.zeros(100), step=0)


def test_resumed_oracle_fit_follows_the_uninterrupted_trajectory(tmp_path):
    """Six Adam steps of the oracle's fit loop with the state held in FP32
    (as the kernels hold it) against three steps, a checkpoint, a load and
    three more steps: bit-identical parameters, moments and losses."""
    R, J = 4, 2000
    qo = synth.sample_batch(synth.sphere(0.5), 2 * J, seed=7)
    p0 = synth.init_params(R, seed=8)
    lb = float(np.float32(oracle.default_log_beta0(R)))
    f32 = lambda a: a.astype(np.float32).astype(np.float64)

    def run(p, m, v, steps, first):
        losses = []
        for s in range(first, first + steps):
            b = (s - 1) % 2
            p, m, v, L, _ = oracle.fit_step(p, m, v, s, qo[b * J:(b + 1) * J], R, loss=oracle.MSE, lr=1e-2,
                                            log_beta0=lb)
            p, m, v = f32(p), f32(m), f32(v)
            losses.append(L)
        return p, m, v, losses

    z = np.zeros_like(p0, dtype=np.float64)
    pa, ma, va, la = run(f32(p0), z, z, 6, 1)
    pb, mb, vb, lb1 = run(f32(p0), z, z, 3, 1)
    path = tmp_path / "r.ckp"
    api.save_checkpoint(path, *(torch.from_numpy(a.astype(np.float32).reshape(-1)) for a in (pb, mb, vb)), step=3,
                        log_beta0=lb, loss="mse", lr=1e-2)
    c = api.load_checkpoint(path, device="cpu")
    assert c["step"] == 3
    pc, mc, vc = (c[k].numpy().astype(np.float64).reshape(p0.shape) for k in ("params", "m", "v"))
    pr, mr, vr, lb2 = run(pc, mc, vc, 3, c["step"] + 1)
    np.testing.assert_array_equal(pr, pa)
    np.testing.assert_array_equal(mr, ma)
    np.testing.assert_array_equal(vr, va)
    assert lb1 + lb2 == la


def test_concurrent_saves_to_one_path_leave_one_complete_file(tmp_path):
    """Threads of one process saving to the same path at once use distinct
    temporary names: every save succeeds, the file left is one of the
    complete checkpoints, and no temporary file remains."""
    import threading
    n = 8 ** 3 * 13
    states = [_state(n, 100 + k) for k in range(6)]
    path = tmp_path / "same.ckp"
    errors = []

    def save(k):
        try:
            for _ in range(5):
                api.save_checkpoint(path, *states[k], step=k)
        except Exception as e:   # noqa: BLE001 - reported below
            errors.append(e)

    threads = [threading.Thread(target=save, args=(k,)) for k in range(len(states))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    c = api.load_checkpoint(path, device="cpu")
    k = c["step"]
    for name, t in zip(("params", "m", "v"), states[k]):
        assert torch.equal(c[name], t)
    assert sorted(os.listdir(tmp_path)) == ["same.ckp"]
