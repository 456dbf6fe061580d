"""Host-side checks of the C ABI: the library builds for sm_103a, loads without
a GPU, exports every symbol include/efunc.h declares, and validates arguments
on the host (nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest
import torch

from paper_2505_21319_gb300 import _binding as B

# Tests that pass made-up device addresses to reach the host-side checks run
# only where no CUDA device is visible: if a check ever regressed, the call
# would enqueue work on those addresses, which must never happen on a GPU.
fake_pointers = pytest.mark.skipif(torch.cuda.is_available(),
                                   reason="made-up device pointers are only passed where no GPU is visible")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "efunc.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(efunc_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_hot_path_calls():
    names = declared_functions()
    for n in ("efunc_forward", "efunc_backward", "efunc_adam_step", "efunc_fit", "efunc_workspace_bytes",
              "efunc_status_str", "efunc_cell_sort"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in B.SIGNATURES, f"binding lacks {name}"
    assert set(B.SIGNATURES) == set(declared_functions())


def test_host_helpers(lib):
    n0 = lib.efunc_launch_count()   # launches of earlier tests in this process
    assert lib.efunc_param_count(32) == 32 ** 3 * 13 == 425984
    assert lib.efunc_param_count(0) == -1 and lib.efunc_param_count(257) == -1
    assert abs(lib.efunc_default_log_beta0(32) - 7.0) < 1e-6
    assert abs(lib.efunc_default_log_beta0(64) - (7.0 + 2 * 0.6931471805599453)) < 1e-6
    for code in range(6):
        assert lib.efunc_status_str(code)
    assert lib.efunc_status_str(99) == b"unknown status"
    assert lib.efunc_last_cuda_error() == 0
    assert lib.efunc_cuda_error_name(1) == b"cudaErrorInvalidValue"
    g = B.Grid(32, 2, 7.0)
    n1 = lib.efunc_workspace_bytes(ctypes.byref(g), 1 << 22)
    n2 = lib.efunc_workspace_bytes(ctypes.byref(g), 1 << 10)
    assert n1 > n2 > 0 and n1 % 256 == 0
    assert lib.efunc_workspace_bytes(ctypes.byref(B.Grid(0, 2, 7.0)), 10) == 0
    assert lib.efunc_workspace_bytes(ctypes.byref(g), -1) == 0
    # the pipelined fit's second sort buffer: about 20 bytes per query more
    nf = lib.efunc_fit_workspace_bytes(ctypes.byref(g), 1 << 22)
    assert nf > n1 and nf - n1 >= 20 * (1 << 22) and nf % 256 == 0
    assert lib.efunc_fit_workspace_bytes(ctypes.byref(B.Grid(0, 2, 7.0)), 10) == 0
    # the sort / forward / backward layout leaves out the gradient grid and
    # the two host-batch staging buffers (32 bytes per query, 52 R^3 bytes)
    ne = lib.efunc_eval_workspace_bytes(ctypes.byref(g), 1 << 22)
    assert 0 < ne < n1 and n1 - ne >= 32 * (1 << 22) + 52 * 32 ** 3 and ne % 256 == 0
    assert lib.efunc_eval_workspace_bytes(ctypes.byref(B.Grid(0, 2, 7.0)), 10) == 0
    assert lib.efunc_eval_workspace_bytes(ctypes.byref(g), -1) == 0
    assert lib.efunc_launch_count() == n0


def _fwd(lib, grid, J=16, stride=3, ws=1 << 30, ws_bytes=None, params=4096, q=8192, O=12288):
    g = ctypes.byref(grid) if grid is not None else None
    if ws_bytes is None:
        ws_bytes = 1 << 40
    return lib.efunc_forward(g, params, q, J, stride, O, None, None, ws, ws_bytes, None)


@fake_pointers
def test_argument_validation_enqueues_nothing(lib):
    """Invalid arguments are rejected on the host (fake, never dereferenced
    pointers are enough to reach every check)."""
    n0 = lib.efunc_launch_count()   # launches of earlier tests in this process
    ok = B.Grid(8, 2, 7.0)
    assert _fwd(lib, None) == 1
    assert _fwd(lib, B.Grid(0, 2, 7.0)) == 1
    assert _fwd(lib, B.Grid(300, 2, 7.0)) == 1
    assert _fwd(lib, B.Grid(8, 3, 7.0)) == 5
    assert _fwd(lib, B.Grid(8, 2, float("nan"))) == 4
    assert _fwd(lib, B.Grid(8, 2, float("inf"))) == 4
    assert _fwd(lib, ok, J=-1) == 1
    assert _fwd(lib, ok, J=(1 << 30) + 1) == 1
    assert _fwd(lib, ok, stride=2) == 1
    assert _fwd(lib, ok, params=None) == 1
    assert _fwd(lib, ok, q=None) == 1
    assert _fwd(lib, ok, ws=None) == 3
    assert _fwd(lib, ok, ws=(1 << 30) + 8) == 3          # misaligned
    assert _fwd(lib, ok, ws_bytes=100) == 3              # too small
    ne = lib.efunc_eval_workspace_bytes(ctypes.byref(ok), 16)
    assert _fwd(lib, ok, ws_bytes=ne - 256) == 3         # one region short of the forward's layout
    assert _fwd(lib, ok, J=0) == 0                       # empty batch: nothing to do
    assert lib.efunc_launch_count() == n0
    # backward, cell sort, Adam, fit
    assert lib.efunc_backward(ctypes.byref(ok), 4096, 8192, 16, 3, 4096, None, None, 1 << 30, 1 << 40, None) == 1
    assert lib.efunc_backward(ctypes.byref(ok), 4096, 8192, 0, 3, None, 4096, None, 1 << 30, 1 << 40, None) == 0
    assert lib.efunc_cell_sort(ctypes.byref(ok), 4096, 16, 3, 8200, 4096, 1 << 30, 1 << 40, None) == 1  # misaligned out
    ad = B.Adam(1e-3, 0.9, 0.999, 1e-8, 0.0, 0)
    assert lib.efunc_adam_step(ctypes.byref(ad), 10, 16, 32, 48, 64, 0, None) == 1           # step 0
    assert lib.efunc_adam_step(ctypes.byref(B.Adam(float("nan"), 0.9, 0.999, 1e-8, 0, 0)), 10, 16, 32, 48, 64, 1,
                               None) == 4
    assert lib.efunc_adam_step(ctypes.byref(B.Adam(1e-3, 1.0, 0.999, 1e-8, 0, 0)), 10, 16, 32, 48, 64, 1, None) == 1
    assert lib.efunc_adam_step(ctypes.byref(ad), 0, None, None, None, None, 1, None) == 0
    assert lib.efunc_fit(ctypes.byref(ok), ctypes.byref(ad), 2, 0.0, 16, 32, 48, 64, 10, 1, 1, 0, None, 1 << 30,
                         1 << 40, None) == 1                                                # bad loss kind
    assert lib.efunc_fit(ctypes.byref(ok), ctypes.byref(ad), 0, 0.0, 16, 32, 48, 64, 10, 0, 1, 0, None, 1 << 30,
                         1 << 40, None) == 1                                                # no batches
    assert lib.efunc_fit(ctypes.byref(ok), ctypes.byref(ad), 0, -1.0, 16, 32, 48, 64, 10, 1, 1, 0, None, 1 << 30,
                         1 << 40, None) == 1                                                # negative weight
    assert lib.efunc_fit(ctypes.byref(ok), ctypes.byref(ad), 0, float("nan"), 16, 32, 48, 64, 10, 1, 1, 0, None,
                         1 << 30, 1 << 40, None) == 4                                       # non-finite weight
    assert lib.efunc_fit(ctypes.byref(ok), ctypes.byref(ad), 0, 0.0, 16, 32, 48, 64, 10, 1, 0, 0, None, 1 << 30,
                         1 << 40, None) == 0                                                # zero steps
    assert lib.efunc_fit(ctypes.byref(ok), ctypes.byref(ad), 0, 0.0, 16, 32, 48, 64, 10, 1, 1, 0, None, 1 << 30,
                         lib.efunc_eval_workspace_bytes(ctypes.byref(ok), 10), None) == 3   # no gradient region
    assert lib.efunc_backward_grad(ctypes.byref(ok), 4096, 8192, 16, 3, None, None, 4096, 1 << 30, 1 << 40,
                                   None) == 1                                               # neither gO nor gG
    # the graph-replayed fit: the same checks, its whole workspace, device batches, at most 64 batches
    fg = lib.efunc_fit_graph
    wsf = lib.efunc_fit_workspace_bytes(ctypes.byref(ok), 16)
    assert fg(ctypes.byref(ok), ctypes.byref(ad), 2, 0.0, 16, 32, 48, 64, 16, 1, 1, 0, None, 1 << 30, wsf,
              None) == 1                                                                    # bad loss kind
    assert fg(ctypes.byref(ok), ctypes.byref(ad), 0, float("inf"), 16, 32, 48, 64, 16, 1, 1, 0, None, 1 << 30, wsf,
              None) == 4
    assert fg(ctypes.byref(ok), ctypes.byref(ad), 0, 0.0, 16, 32, 48, 64, 16, 0, 1, 0, None, 1 << 30, wsf,
              None) == 1                                                                    # no batches
    assert fg(ctypes.byref(ok), ctypes.byref(ad), 0, 0.0, 16, 32, 48, 64, 16, 65, 1, 0, None, 1 << 30, wsf,
              None) == 1                                                                    # period too long
    assert fg(ctypes.byref(ok), ctypes.byref(ad), 0, 0.0, 16, 32, 48, 64, 16, 1, 1, 0, None, 1 << 30, wsf - 256,
              None) == 3                                                                    # no second sort buffer
    assert fg(ctypes.byref(ok), ctypes.byref(ad), 0, 0.0, 16, 32, 48, 64, 16, 1, 1, 0, None, (1 << 30) + 64, wsf,
              None) == 3                                                                    # misaligned
    assert fg(ctypes.byref(ok), ctypes.byref(ad), 0, 0.0, 16, 32, 48, 64, 16, 1, 0, 0, None, 1 << 30, wsf,
              None) == 0                                                                    # zero steps
    assert fg(ctypes.byref(ok), ctypes.byref(ad), 0, 0.0, 16, 32, 48, 64, 16, 1, 1, 0, None, 1 << 30, wsf,
              None) == 1                                                                    # not device memory
    assert lib.efunc_mean_shift_init(ctypes.byref(ok), 4096, 0, 100.0, 8192, None) == 1       # no points
    assert lib.efunc_mean_shift_init(ctypes.byref(ok), 4096, (1 << 30) + 1, 100.0, 8192, None) == 1
    assert lib.efunc_mean_shift_init(ctypes.byref(ok), 4096, 10, 0.0, 8192, None) == 1        # bandwidth 0
    assert lib.efunc_mean_shift_init(ctypes.byref(ok), 4096, 10, -1.0, 8192, None) == 1
    assert lib.efunc_mean_shift_init(ctypes.byref(ok), 4096, 10, float("inf"), 8192, None) == 4
    assert lib.efunc_mean_shift_init(ctypes.byref(ok), None, 10, 100.0, 8192, None) == 1
    assert lib.efunc_mean_shift_init(ctypes.byref(B.Grid(0, 2, 7.0)), 4096, 10, 100.0, 8192, None) == 1
    assert lib.efunc_launch_count() == n0


@fake_pointers
def test_variant_helpers_and_validation(lib):
    """Channel counts of the ablation variants and host-side rejection of
    invalid variant requests (nothing launches)."""
    n0 = lib.efunc_launch_count()   # launches of earlier tests in this process
    from paper_2505_21319_gb300 import api
    for name, (sets, deg, learn) in api.VARIANTS.items():
        ch = lib.efunc_variant_channels(ctypes.byref(B.Variant(sets, deg, learn)))
        assert ch == {"G-1": 1, "G-2": 4, "G-3": 10, "G-4": 20, "G-5": 2, "G-6": 5, "G-7": 11, "G-8": 21,
                      "Full-1": 8, "Full-3": 13}[name]
    for bad in ((0, 1, 1), (4, 1, 1), (1, 4, 1), (1, -1, 0), (3, 1, 2)):
        assert lib.efunc_variant_channels(ctypes.byref(B.Variant(*bad))) == -1
    assert lib.efunc_variant_channels(None) == -1
    g = B.Grid(8, 2, 7.0)
    v = B.Variant(3, 3, 1)
    big = lib.efunc_variant_workspace_bytes(ctypes.byref(g), ctypes.byref(v), 1 << 16)
    small = lib.efunc_variant_workspace_bytes(ctypes.byref(g), ctypes.byref(B.Variant(1, 0, 0)), 1 << 16)
    assert big > small > 0 and big % 256 == 0
    assert lib.efunc_variant_workspace_bytes(ctypes.byref(g), ctypes.byref(B.Variant(0, 1, 1)), 10) == 0
    fwd = lib.efunc_variant_forward
    assert fwd(ctypes.byref(g), ctypes.byref(B.Variant(5, 1, 1)), 4096, 8192, 16, 3, 12288, None, 1 << 30, 1 << 40,
               None) == 1                                                                   # bad variant
    assert fwd(ctypes.byref(g), ctypes.byref(v), 4096, 8192, 16, 3, 12288, None, 1 << 30, 100, None) == 3
    assert fwd(ctypes.byref(g), ctypes.byref(v), 4096, 8192, 0, 3, None, None, 1 << 30, 1 << 40, None) == 0
    assert lib.efunc_variant_backward(ctypes.byref(g), ctypes.byref(v), 4096, 8192, 16, 3, None, 4096, 1 << 30,
                                      1 << 40, None) == 1                                    # no gO
    ad = B.Adam(1e-3, 0.9, 0.999, 1e-8, 0.0, 0)
    assert lib.efunc_variant_fit(ctypes.byref(g), ctypes.byref(v), ctypes.byref(ad), 0, 16, 32, 48, 64, 10, 0, 1, 0,
                                 None, 1 << 30, 1 << 40, None) == 1                          # no batches
    # the variant fit needs its whole workspace (second sort buffer) and device batches
    v1 = B.Variant(1, 1, 1)
    wsv = lib.efunc_variant_workspace_bytes(ctypes.byref(g), ctypes.byref(v1), 16)
    assert lib.efunc_variant_fit(ctypes.byref(g), ctypes.byref(v1), ctypes.byref(ad), 0, 16, 32, 48, 64, 16, 1, 1, 0,
                                 None, 1 << 30, wsv - 256, None) == 3
    assert lib.efunc_variant_fit(ctypes.byref(g), ctypes.byref(v1), ctypes.byref(ad), 0, 16, 32, 48, 64, 16, 1, 1, 0,
                                 None, 1 << 30, wsv, None) == 1                              # not device memory
    assert lib.efunc_launch_count() == n0


@fake_pointers
def test_cosine_helpers_and_validation(lib):
    n0 = lib.efunc_launch_count()   # launches of earlier tests in this process
    g = B.Grid(16, 2, 7.0)
    n1 = lib.efunc_cosine_workspace_bytes(ctypes.byref(g), 1, 1 << 16)
    n8 = lib.efunc_cosine_workspace_bytes(ctypes.byref(g), 8, 1 << 16)
    assert n8 > n1 > 0 and n8 % 256 == 0
    assert lib.efunc_cosine_workspace_bytes(ctypes.byref(g), 0, 10) == 0
    assert lib.efunc_cosine_workspace_bytes(ctypes.byref(g), 17, 10) == 0
    assert lib.efunc_cosine_forward(ctypes.byref(g), 0, 4096, 8192, 16, 3, 12288, 1 << 30, 1 << 40, None) == 1
    assert lib.efunc_cosine_forward(ctypes.byref(g), 4, 4096, 8192, 16, 3, 12288, 1 << 30, 100, None) == 3
    assert lib.efunc_cosine_forward(ctypes.byref(g), 4, 4096, 8192, 0, 3, None, 1 << 30, 1 << 40, None) == 0
    assert lib.efunc_cosine_backward(ctypes.byref(g), 4, 4096, 8192, 16, 3, None, 4096, 1 << 30, 1 << 40,
                                     None) == 1
    ad = B.Adam(1e-3, 0.9, 0.999, 1e-8, 0.0, 0)
    assert lib.efunc_cosine_fit(ctypes.byref(g), 4, ctypes.byref(ad), 3, 16, 32, 48, 64, 10, 1, 1, 0, None, 1 << 30,
                                1 << 40, None) == 1                                          # bad loss kind
    wsc = lib.efunc_cosine_workspace_bytes(ctypes.byref(g), 4, 16)
    assert lib.efunc_cosine_fit(ctypes.byref(g), 4, ctypes.byref(ad), 0, 16, 32, 48, 64, 16, 1, 1, 0, None, 1 << 30,
                                wsc - 256, None) == 3                                        # workspace too small
    assert lib.efunc_launch_count() == n0


def test_profile_api_without_gpu(lib):
    ms, cnt = ctypes.c_double(1.0), ctypes.c_int64(1)
    lib.efunc_profile_reset()
    assert lib.efunc_profile_read(b"fused_fit", ctypes.byref(ms), ctypes.byref(cnt)) == 0
    assert ms.value == 0.0 and cnt.value == 0
    assert lib.efunc_profile_read(b"nope", ctypes.byref(ms), ctypes.byref(cnt)) == -1


def _shapes(*rj):
    return (B.Shape * len(rj))(*[B.Shape(R, 7.0, J) for R, J in rj])


def test_batched_helpers(lib):
    sh = _shapes((16, 1000), (32, 5000), (64, 1 << 14))
    assert lib.efunc_batched_param_count(sh, 3) == 13 * (16 ** 3 + 32 ** 3 + 64 ** 3)
    assert lib.efunc_batched_query_count(sh, 3) == 1000 + 5000 + (1 << 14)
    n3 = lib.efunc_batched_workspace_bytes(sh, 3)
    n2 = lib.efunc_batched_workspace_bytes(sh, 2)
    assert n3 > n2 > 0 and n3 % 256 == 0
    for bad in (_shapes((0, 10)), _shapes((257, 10)), _shapes((8, 0)), _shapes((8, (1 << 30) + 1))):
        assert lib.efunc_batched_param_count(bad, 1) == -1
        assert lib.efunc_batched_workspace_bytes(bad, 1) == 0
    assert lib.efunc_batched_param_count(sh, 0) == -1
    assert lib.efunc_batched_param_count(sh, 1025) == -1
    t = B.Tuning()
    lib.efunc_default_tuning(ctypes.byref(t))
    assert (t.chunk, t.lanes2_max, t.lanes4_max, t.sort_blocks, t.group_max) == (256, 64, 32, 8, 128)


@fake_pointers
def test_batched_validation_enqueues_nothing(lib):
    n0 = lib.efunc_launch_count()
    sh = _shapes((8, 100), (4, 50))
    ad = B.Adam(1e-3, 0.9, 0.999, 1e-8, 0.0, 0)
    ws = lib.efunc_batched_workspace_bytes(sh, 2)
    f = lib.efunc_fit_batched
    args = lambda **k: dict(dict(shapes=sh, S=2, loss=0, nb=1, steps=1, tuning=None, graph=0, ws=1 << 30,
                                 wsb=ws), **k)

    def call(**k):
        a = args(**k)
        return f(a["shapes"], a["S"], ctypes.byref(ad), a["loss"], 16, 32, 48, 64, a["nb"], a["steps"], 0, None,
                 a["tuning"], a["graph"], a["ws"], a["wsb"], None)
    assert call(loss=2) == 1                       # bad loss kind
    assert call(nb=0) == 1                         # no batches
    assert call(nb=65) == 1
    assert call(graph=2) == 1
    assert call(S=0) == 1
    assert call(shapes=_shapes((0, 10)), S=1) == 1
    assert call(tuning=ctypes.byref(B.Tuning(16, 64, 32, 8))) == 1    # chunk below 32
    assert call(tuning=ctypes.byref(B.Tuning(256, 32, 64, 8))) == 1   # lanes4 > lanes2
    assert call(tuning=ctypes.byref(B.Tuning(256, 64, 32, 0))) == 1   # no sort blocks
    assert call(tuning=ctypes.byref(B.Tuning(256, 64, 32, 8, 300))) == 1   # octets above an item's capacity
    assert call(wsb=ws - 256) == 3
    assert call(ws=(1 << 30) + 64) == 3
    assert call(steps=0) == 0
    assert call() == 1                             # batches not in device memory
    out = lib.efunc_eval_batched(sh, 2, 16, 32, None, None, 1 << 30, ws, None)
    assert out == 1
    assert lib.efunc_tune_batched(sh, 2, 0, 16, 32, 48, 64, 1, 0, ctypes.byref(B.Tuning()), None, 1 << 30, ws,
                                  None) == 1       # no trial steps
    assert lib.efunc_launch_count() == n0


def test_noalloc_capacities_in_the_header(lib):
    """The capacities the header states for efunc_forward_noalloc follow from
    the forward's workspace layout and the fixed 32 MiB array: each is the
    largest J whose efunc_eval_workspace_bytes fits (host arithmetic only)."""
    src = open(HEADER).read()
    m = re.search(r"up to ([\d,]+) queries at R = 32, ([\d,]+) at R = 16 and ([\d,]+) at\s*\*\s*R = 64", src)
    assert m, "capacity sentence not found in efunc.h"
    stated = {32: int(m.group(1).replace(",", "")), 16: int(m.group(2).replace(",", "")),
              64: int(m.group(3).replace(",", ""))}
    cap = 32 << 20
    for R, J in stated.items():
        g = B.Grid(R, 2, float(lib.efunc_default_log_beta0(R)))
        assert 0 < lib.efunc_eval_workspace_bytes(ctypes.byref(g), J) <= cap, R
        assert lib.efunc_eval_workspace_bytes(ctypes.byref(g), J + 1) > cap, R
