"""The bounds-check build (lib/libefunc_debug.so, -DEFUNC_DEBUG_BOUNDS).

CPU: it builds for sm_103a and exports every symbol of include/efunc.h; the
normal build answers efunc_debug_bounds with EFUNC_ERR_UNSUPPORTED.
GPU (child process with EFUNC_DEBUG_BOUNDS=1): forward, backward, the
pipelined and in-line fits, a fit with grouped sparse octets, the batched fit
and the evaluation run with every index check of the kernels on, record no
failing check, and the forward equals the normal build's bit for bit."""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2505_21319_gb300 import _binding as B
from paper_2505_21319_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
from test_abi import declared_functions  # noqa: E402


def test_debug_build_exports_every_declared_symbol():
    path = _build.build(debug=True)
    assert path.endswith("libefunc_debug.so")
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_normal_build_has_no_bounds_flag(lib):
    code = ctypes.c_int32(7)
    assert lib.efunc_debug_bounds(ctypes.byref(code)) == 5   # EFUNC_ERR_UNSUPPORTED
    assert code.value == 0
    assert lib.efunc_debug_bounds(None) == 1                 # EFUNC_ERR_ARG


CHILD = r"""
import json, sys, numpy as np, torch
sys.path.insert(0, ROOT)
from paper_2505_21319_gb300 import api, synth
dev = torch.device("cuda:0")
out = {}
assert api.debug_bounds() == 0
for R, J in ((8, 5003), (16, 65536), (32, 1 << 18)):
    p = torch.from_numpy(synth.random_params(R, seed=R)).to(dev)
    qo = torch.from_numpy(synth.sample_batch(synth.random_union(R), J, seed=R)).to(dev)
    O = api.efunc_forward(p, qo[:, :3].contiguous())
    g = api.efunc_backward(p, qo, torch.full((J,), 1.0 / J, device=dev))
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    api.efunc_fit(p, m, v, qo, steps=3)                       # in line or pipelined, grouped at 32^3 x 2^18
    api.efunc_fit(p, m, v, torch.cat([qo, qo.flip(0)]), steps=4, J=J, n_batches=2)
    api.efunc_eval_loss(p, qo)
    torch.cuda.synchronize()
    out[f"{R}"] = {"code": api.debug_bounds(), "O": O.cpu().numpy().tolist() if J < 6000 else None}
b = api.Batch([16, 32, 64], [3000, 1 << 16, 1 << 17], device=dev)
rows = torch.cat([synth.sample_batch_torch(synth.random_union(s), J, seed=s, device=dev) for s, J in enumerate(b.Js)])
pb = torch.zeros(b.n_params, device=dev); mb, vb = torch.zeros_like(pb), torch.zeros_like(pb)
b.fit(pb, mb, vb, rows, steps=3, graph=False)
b.eval(pb, rows)
torch.cuda.synchronize()
out["batched"] = {"code": api.debug_bounds()}
print(json.dumps(out))
"""


@pytest.mark.gpu
def test_every_index_check_passes_on_the_hot_path():
    env = dict(os.environ, EFUNC_DEBUG_BOUNDS="1")
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + CHILD], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    for k, v in res.items():
        assert v["code"] == 0, f"bounds check {v['code']} failed in case {k}"
    # the checks change no arithmetic: the forward equals the normal build's
    import torch
    from paper_2505_21319_gb300 import api, synth
    dev = torch.device("cuda:0")
    p = torch.from_numpy(synth.random_params(8, seed=8)).to(dev)
    qo = torch.from_numpy(synth.sample_batch(synth.random_union(8), 5003, seed=8)).to(dev)
    O = api.efunc_forward(p, qo[:, :3].contiguous()).cpu().numpy()
    np.testing.assert_array_equal(O, np.array(res["8"]["O"], dtype=np.float32))
