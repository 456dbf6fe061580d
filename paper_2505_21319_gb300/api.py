"""PyTorch-facing wrappers of the C ABI (same names as include/efunc.h).

PyTorch supplies device memory and the current CUDA stream; every step of the
computation runs in the library's kernels.  Tensors must be CUDA float32 and
contiguous; nothing is copied or converted implicitly.
"""
from __future__ import annotations

import ctypes
import math

import torch

from . import _binding as B

NSLOT = 13


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(device):
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _need(t: torch.Tensor, name: str, numel: int | None = None, dtype=torch.float32):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")


def resolution_of(params: torch.Tensor) -> int:
    n = params.numel() // NSLOT
    R = int(round(n ** (1.0 / 3.0)))
    if R ** 3 * NSLOT != params.numel():
        raise ValueError("params must hold R^3 * 13 floats")
    return R


def default_log_beta0(R: int) -> float:
    return float(B.load().efunc_default_log_beta0(R))


def make_grid(R: int, log_beta0: float | None = None, W: int = 2) -> B.Grid:
    return B.Grid(R, W, default_log_beta0(R) if log_beta0 is None else float(log_beta0))


class Workspace:
    """Grow-only device scratch buffer for one stream's calls."""

    def __init__(self, device=None):
        self.device = torch.device(device or "cuda")
        self.buf = None

    def get(self, grid: B.Grid, J: int, fit: bool = False, eval_only: bool = False) -> tuple[torch.Tensor, int]:
        """fit: the pipelined fit's size; eval_only: the sort / forward /
        backward size; neither: the in-line fit's size."""
        lib = B.load()
        query = (lib.efunc_fit_workspace_bytes if fit else
                 lib.efunc_eval_workspace_bytes if eval_only else lib.efunc_workspace_bytes)
        n = int(query(ctypes.byref(grid), int(J)))
        if n == 0:
            raise ValueError("invalid grid or query count")
        if self.buf is None or self.buf.numel() < n:
            self.buf = torch.empty(n, dtype=torch.uint8, device=self.device)
        return self.buf, n


_default_ws: dict = {}


def _workspace(device, ws: Workspace | None) -> Workspace:
    if ws is not None:
        return ws
    key = torch.device(device).index if torch.device(device).index is not None else torch.cuda.current_device()
    if key not in _default_ws:
        _default_ws[key] = Workspace(torch.device("cuda", key))
    return _default_ws[key]


def _queries(q: torch.Tensor, dtype=torch.float32):
    _need(q, "q", dtype=dtype)
    if q.dim() != 2 or q.shape[1] not in (3, 4):
        raise ValueError("q must be (J, 3) or (J, 4)")
    return q.shape[0], q.shape[1]


def efunc_cell_sort(q: torch.Tensor, R: int, ws: Workspace | None = None):
    """Cell-sorted copy of the queries (J, 4) and the permutation (J,) int32."""
    J, stride = _queries(q)
    grid = make_grid(R)
    out = torch.empty((J, 4), dtype=torch.float32, device=q.device)
    perm = torch.empty(J, dtype=torch.int32, device=q.device)
    buf, n = _workspace(q.device, ws).get(grid, J, eval_only=True)
    B.check("efunc_cell_sort", B.load().efunc_cell_sort(ctypes.byref(grid), _ptr(q), J, stride, _ptr(out),
                                                        _ptr(perm), _ptr(buf), n, _stream(q.device)))
    return out, perm


def efunc_forward(params: torch.Tensor, q: torch.Tensor, log_beta0: float | None = None, want_lse: bool = False,
                  want_dq: bool = False, ws: Workspace | None = None):
    """O(q) (Algorithm 1, Eq. func-offset); optionally lse and dO/dq (Eq. func-normal)."""
    R = resolution_of(params)
    _need(params, "params")
    J, stride = _queries(q)
    grid = make_grid(R, log_beta0)
    O = torch.empty(J, dtype=torch.float32, device=q.device)
    lse = torch.empty(J, dtype=torch.float32, device=q.device) if want_lse else None
    dq = torch.empty((J, 3), dtype=torch.float32, device=q.device) if want_dq else None
    buf, n = _workspace(q.device, ws).get(grid, J, eval_only=True)
    B.check("efunc_forward", B.load().efunc_forward(ctypes.byref(grid), _ptr(params), _ptr(q), J, stride, _ptr(O),
                                                    _ptr(lse), _ptr(dq), _ptr(buf), n, _stream(q.device)))
    out = [O]
    if want_lse:
        out.append(lse)
    if want_dq:
        out.append(dq)
    return out[0] if len(out) == 1 else tuple(out)


def efunc_backward(params: torch.Tensor, q: torch.Tensor, gO: torch.Tensor, grad: torch.Tensor | None = None,
                   want_gq: bool = False, log_beta0: float | None = None, ws: Workspace | None = None):
    """Accumulate dL/dparams into ``grad`` (Algorithm 2); optionally dL/dq."""
    R = resolution_of(params)
    _need(params, "params")
    J, stride = _queries(q)
    _need(gO, "gO", J)
    if grad is None:
        grad = torch.zeros_like(params)
    _need(grad, "grad", params.numel())
    gq = torch.empty((J, 3), dtype=torch.float32, device=q.device) if want_gq else None
    grid = make_grid(R, log_beta0)
    buf, n = _workspace(q.device, ws).get(grid, J, eval_only=True)
    B.check("efunc_backward", B.load().efunc_backward(ctypes.byref(grid), _ptr(params), _ptr(q), J, stride,
                                                      _ptr(gO), _ptr(grad), _ptr(gq), _ptr(buf), n,
                                                      _stream(q.device)))
    return (grad, gq) if want_gq else grad


def efunc_backward_grad(params: torch.Tensor, q: torch.Tensor, gO: torch.Tensor | None, gG: torch.Tensor | None,
                        grad: torch.Tensor | None = None, log_beta0: float | None = None,
                        ws: Workspace | None = None):
    """Accumulate dL/dparams for L = sum gO.O + gG . dO/dq (backward through
    Eq. func-normal, e.g. for an Eikonal loss)."""
    R = resolution_of(params)
    _need(params, "params")
    J, stride = _queries(q)
    if gO is not None:
        _need(gO, "gO", J)
    if gG is not None:
        _need(gG, "gG", 3 * J)
    if grad is None:
        grad = torch.zeros_like(params)
    _need(grad, "grad", params.numel())
    grid = make_grid(R, log_beta0)
    buf, n = _workspace(q.device, ws).get(grid, J, eval_only=True)
    B.check("efunc_backward_grad", B.load().efunc_backward_grad(ctypes.byref(grid), _ptr(params), _ptr(q), J, stride,
                                                                _ptr(gO), _ptr(gG), _ptr(grad), _ptr(buf), n,
                                                                _stream(q.device)))
    return grad


def efunc_eval_loss(params: torch.Tensor, qo: torch.Tensor, log_beta0: float | None = None,
                    ws: Workspace | None = None) -> torch.Tensor:
    """(mean (O - o)^2, mean |O - o|) over rows (x, y, z, target) of ``qo``,
    as a CUDA float32 tensor of 2 (no synchronisation)."""
    R = resolution_of(params)
    _need(params, "params")
    _need(qo, "qo")
    if qo.dim() != 2 or qo.shape[1] != 4 or qo.shape[0] < 1:
        raise ValueError("qo must be (J, 4) with J >= 1")
    J = qo.shape[0]
    grid = make_grid(R, log_beta0)
    out = torch.empty(2, dtype=torch.float32, device=qo.device)
    buf, n = _workspace(qo.device, ws).get(grid, J, eval_only=True)
    B.check("efunc_eval_loss", B.load().efunc_eval_loss(ctypes.byref(grid), _ptr(params), _ptr(qo), J, _ptr(out),
                                                        _ptr(buf), n, _stream(qo.device)))
    return out


def _f64_workspace(device, grid, J):
    n = int(B.load().efunc_f64_workspace_bytes(ctypes.byref(grid), int(J)))
    if n == 0:
        raise ValueError("invalid grid or query count")
    return torch.empty(n, dtype=torch.uint8, device=device), n


def efunc_forward_f64(params: torch.Tensor, q: torch.Tensor, log_beta0: float | None = None, want_lse: bool = False,
                      want_dq: bool = False):
    """The forward in FP64 (float64 params and queries): O, optionally lse and dO/dq."""
    R = resolution_of(params)
    _need(params, "params", dtype=torch.float64)
    J, stride = _queries(q, torch.float64)
    grid = make_grid(R, log_beta0)
    O = torch.empty(J, dtype=torch.float64, device=q.device)
    lse = torch.empty(J, dtype=torch.float64, device=q.device) if want_lse else None
    dq = torch.empty((J, 3), dtype=torch.float64, device=q.device) if want_dq else None
    buf, n = _f64_workspace(q.device, grid, J)
    B.check("efunc_forward_f64", B.load().efunc_forward_f64(ctypes.byref(grid), _ptr(params), _ptr(q), J, stride,
                                                            _ptr(O), _ptr(lse), _ptr(dq), _ptr(buf), n,
                                                            _stream(q.device)))
    out = [O] + ([lse] if want_lse else []) + ([dq] if want_dq else [])
    return out[0] if len(out) == 1 else tuple(out)


def efunc_backward_f64(params: torch.Tensor, q: torch.Tensor, gO: torch.Tensor, grad: torch.Tensor | None = None,
                       want_gq: bool = False, log_beta0: float | None = None):
    """The backward in FP64: accumulates dL/dparams into ``grad``; optionally dL/dq."""
    R = resolution_of(params)
    _need(params, "params", dtype=torch.float64)
    J, stride = _queries(q, torch.float64)
    _need(gO, "gO", J, dtype=torch.float64)
    if grad is None:
        grad = torch.zeros_like(params)
    _need(grad, "grad", params.numel(), dtype=torch.float64)
    gq = torch.empty((J, 3), dtype=torch.float64, device=q.device) if want_gq else None
    grid = make_grid(R, log_beta0)
    buf, n = _f64_workspace(q.device, grid, J)
    B.check("efunc_backward_f64", B.load().efunc_backward_f64(ctypes.byref(grid), _ptr(params), _ptr(q), J, stride,
                                                              _ptr(gO), _ptr(grad), _ptr(gq), _ptr(buf), n,
                                                              _stream(q.device)))
    return (grad, gq) if want_gq else grad


def efunc_mean_shift_init(params: torch.Tensor, pts: torch.Tensor, bandwidth: float = 100.0):
    """Write the mean-shift offsets of Sec. 3.3 into params slots 0..2 (in place)."""
    R = resolution_of(params)
    _need(params, "params")
    _need(pts, "pts")
    if pts.dim() != 2 or pts.shape[1] != 3:
        raise ValueError("pts must be (N, 3)")
    grid = make_grid(R)
    B.check("efunc_mean_shift_init", B.load().efunc_mean_shift_init(ctypes.byref(grid), _ptr(pts), pts.shape[0],
                                                                    float(bandwidth), _ptr(params),
                                                                    _stream(params.device)))
    return params


# Configurations of Table tab:ablation: (key sets, value degree, learnable scale)
VARIANTS = {
    "G-1": (B.KEYS_GRID, 0, 0), "G-2": (B.KEYS_GRID, 1, 0), "G-3": (B.KEYS_GRID, 2, 0), "G-4": (B.KEYS_GRID, 3, 0),
    "G-5": (B.KEYS_GRID, 0, 1), "G-6": (B.KEYS_GRID, 1, 1), "G-7": (B.KEYS_GRID, 2, 1), "G-8": (B.KEYS_GRID, 3, 1),
    "Full-1": (B.KEYS_OFFSET, 1, 1), "Full-3": (B.KEYS_BOTH, 1, 1),
}


def make_variant(variant) -> B.Variant:
    """A Variant from a Table tab:ablation name or a (sets, degree, learn_scale) tuple."""
    if isinstance(variant, B.Variant):
        return variant
    sets, deg, learn = VARIANTS[variant] if isinstance(variant, str) else variant
    return B.Variant(int(sets), int(deg), int(learn))


def variant_channels(variant) -> int:
    ch = int(B.load().efunc_variant_channels(ctypes.byref(make_variant(variant))))
    if ch < 0:
        raise ValueError(f"invalid variant {variant}")
    return ch


class VariantWorkspace(Workspace):
    """Grow-only device scratch for the variant calls."""

    def get_variant(self, grid: B.Grid, var: B.Variant, J: int) -> tuple[torch.Tensor, int]:
        n = int(B.load().efunc_variant_workspace_bytes(ctypes.byref(grid), ctypes.byref(var), int(J)))
        if n == 0:
            raise ValueError("invalid grid, variant or query count")
        if self.buf is None or self.buf.numel() < n:
            self.buf = torch.empty(n, dtype=torch.uint8, device=self.device)
        return self.buf, n


_variant_ws: dict = {}


def _vworkspace(device, ws):
    if ws is not None:
        return ws
    key = torch.device(device).index if torch.device(device).index is not None else torch.cuda.current_device()
    if key not in _variant_ws:
        _variant_ws[key] = VariantWorkspace(torch.device("cuda", key))
    return _variant_ws[key]


def _variant_resolution(params, ch):
    n = params.numel() // ch
    R = int(round(n ** (1.0 / 3.0)))
    if R ** 3 * ch != params.numel():
        raise ValueError(f"params must hold R^3 * {ch} floats")
    return R


def efunc_variant_forward(variant, params: torch.Tensor, q: torch.Tensor, log_beta0: float | None = None,
                          want_lse: bool = False, ws=None):
    """O(q) of a Table tab:ablation variant; optionally lse."""
    var = make_variant(variant)
    R = _variant_resolution(params, variant_channels(var))
    _need(params, "params")
    J, stride = _queries(q)
    grid = make_grid(R, log_beta0)
    O = torch.empty(J, dtype=torch.float32, device=q.device)
    lse = torch.empty(J, dtype=torch.float32, device=q.device) if want_lse else None
    buf, n = _vworkspace(q.device, ws).get_variant(grid, var, J)
    B.check("efunc_variant_forward", B.load().efunc_variant_forward(
        ctypes.byref(grid), ctypes.byref(var), _ptr(params), _ptr(q), J, stride, _ptr(O), _ptr(lse), _ptr(buf), n,
        _stream(q.device)))
    return (O, lse) if want_lse else O


def efunc_variant_backward(variant, params: torch.Tensor, q: torch.Tensor, gO: torch.Tensor,
                           grad: torch.Tensor | None = None, log_beta0: float | None = None, ws=None):
    """Accumulate sum_j gO_j dO_j/dparams of a variant into ``grad``."""
    var = make_variant(variant)
    R = _variant_resolution(params, variant_channels(var))
    _need(params, "params")
    J, stride = _queries(q)
    _need(gO, "gO", J)
    if grad is None:
        grad = torch.zeros_like(params)
    _need(grad, "grad", params.numel())
    grid = make_grid(R, log_beta0)
    buf, n = _vworkspace(q.device, ws).get_variant(grid, var, J)
    B.check("efunc_variant_backward", B.load().efunc_variant_backward(
        ctypes.byref(grid), ctypes.byref(var), _ptr(params), _ptr(q), J, stride, _ptr(gO), _ptr(grad), _ptr(buf), n,
        _stream(q.device)))
    return grad


def efunc_variant_fit(variant, params, m, v, qo, steps: int, J: int | None = None, n_batches: int = 1,
                      step0: int = 0, loss: str = "l1", stats=None, log_beta0: float | None = None, ws=None,
                      **adam_kw):
    """Fitting loop (Sec. 3.4) of a variant on device batches of (x, y, z, target) rows."""
    var = make_variant(variant)
    R = _variant_resolution(params, variant_channels(var))
    for t, nm in ((params, "params"), (m, "m"), (v, "v")):
        _need(t, nm, params.numel())
    _need(qo, "qo")
    if qo.dim() != 2 or qo.shape[1] != 4:
        raise ValueError("qo must be (n_batches*J, 4)")
    if J is None:
        J = qo.shape[0] // n_batches
    if J * n_batches != qo.shape[0]:
        raise ValueError("qo must hold n_batches * J rows")
    if stats is not None:
        _need(stats, "stats")
        if stats.numel() < 2 * steps:
            raise ValueError("stats must hold at least 2*steps floats")
    grid = make_grid(R, log_beta0)
    ad = make_adam(**adam_kw)
    buf, n = _vworkspace(params.device, ws).get_variant(grid, var, J)
    lk = {"l1": B.LOSS_L1, "mse": B.LOSS_MSE}[loss]
    B.check("efunc_variant_fit", B.load().efunc_variant_fit(
        ctypes.byref(grid), ctypes.byref(var), ctypes.byref(ad), lk, _ptr(params), _ptr(m), _ptr(v), _ptr(qo), J,
        n_batches, steps, step0, _ptr(stats), _ptr(buf), n, _stream(params.device)))


class CosineWorkspace(Workspace):
    """Grow-only device scratch for the cosine-series calls."""

    def get_cosine(self, grid: B.Grid, bands: int, J: int) -> tuple[torch.Tensor, int]:
        n = int(B.load().efunc_cosine_workspace_bytes(ctypes.byref(grid), int(bands), int(J)))
        if n == 0:
            raise ValueError("invalid grid, band count or query count")
        if self.buf is None or self.buf.numel() < n:
            self.buf = torch.empty(n, dtype=torch.uint8, device=self.device)
        return self.buf, n


_cosine_ws: dict = {}


def _cworkspace(device, ws):
    if ws is not None:
        return ws
    key = torch.device(device).index if torch.device(device).index is not None else torch.cuda.current_device()
    if key not in _cosine_ws:
        _cosine_ws[key] = CosineWorkspace(torch.device("cuda", key))
    return _cosine_ws[key]


def _cosine_resolution(params, bands):
    return _variant_resolution(params, 5 * bands)


def efunc_cosine_forward(bands: int, params: torch.Tensor, q: torch.Tensor, log_beta0: float | None = None,
                         ws=None):
    """S(q) of the cosine-series decomposition (Sec. 4.4); params (B, R^3, 5)."""
    R = _cosine_resolution(params, bands)
    _need(params, "params")
    J, stride = _queries(q)
    grid = make_grid(R, log_beta0)
    S = torch.empty(J, dtype=torch.float32, device=q.device)
    buf, n = _cworkspace(q.device, ws).get_cosine(grid, bands, J)
    B.check("efunc_cosine_forward", B.load().efunc_cosine_forward(
        ctypes.byref(grid), int(bands), _ptr(params), _ptr(q), J, stride, _ptr(S), _ptr(buf), n, _stream(q.device)))
    return S


def efunc_cosine_backward(bands: int, params: torch.Tensor, q: torch.Tensor, gS: torch.Tensor,
                          grad: torch.Tensor | None = None, log_beta0: float | None = None, ws=None):
    """Accumulate sum_j gS_j dS_j/dparams into ``grad``."""
    R = _cosine_resolution(params, bands)
    _need(params, "params")
    J, stride = _queries(q)
    _need(gS, "gS", J)
    if grad is None:
        grad = torch.zeros_like(params)
    _need(grad, "grad", params.numel())
    grid = make_grid(R, log_beta0)
    buf, n = _cworkspace(q.device, ws).get_cosine(grid, bands, J)
    B.check("efunc_cosine_backward", B.load().efunc_cosine_backward(
        ctypes.byref(grid), int(bands), _ptr(params), _ptr(q), J, stride, _ptr(gS), _ptr(grad), _ptr(buf), n,
        _stream(q.device)))
    return grad


def efunc_cosine_fit(bands: int, params, m, v, qo, steps: int, J: int | None = None, n_batches: int = 1,
                     step0: int = 0, loss: str = "l1", stats=None, log_beta0: float | None = None, ws=None,
                     **adam_kw):
    """Fitting loop of S (Sec. 4.4) on device batches of (x, y, z, target) rows."""
    R = _cosine_resolution(params, bands)
    for t, nm in ((params, "params"), (m, "m"), (v, "v")):
        _need(t, nm, params.numel())
    _need(qo, "qo")
    if qo.dim() != 2 or qo.shape[1] != 4:
        raise ValueError("qo must be (n_batches*J, 4)")
    if J is None:
        J = qo.shape[0] // n_batches
    if J * n_batches != qo.shape[0]:
        raise ValueError("qo must hold n_batches * J rows")
    if stats is not None:
        _need(stats, "stats")
    grid = make_grid(R, log_beta0)
    ad = make_adam(**adam_kw)
    buf, n = _cworkspace(params.device, ws).get_cosine(grid, bands, J)
    lk = {"l1": B.LOSS_L1, "mse": B.LOSS_MSE}[loss]
    B.check("efunc_cosine_fit", B.load().efunc_cosine_fit(
        ctypes.byref(grid), int(bands), ctypes.byref(ad), lk, _ptr(params), _ptr(m), _ptr(v), _ptr(qo), J,
        n_batches, steps, step0, _ptr(stats), _ptr(buf), n, _stream(params.device)))


def make_adam(lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, decoupled=False) -> B.Adam:
    return B.Adam(lr, beta1, beta2, eps, weight_decay, int(bool(decoupled)))


def _host_f32(t: torch.Tensor, n: int, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or t.numel() != n:
        raise ValueError(f"{name} must be a tensor of {n} floats")
    return t.detach().to("cpu", torch.float32).contiguous()


def save_checkpoint(path: str, params: torch.Tensor, m: torch.Tensor, v: torch.Tensor, step: int,
                    channels: int = 13, log_beta0: float | None = None, W: int = 2, seed: int = 0,
                    loss: str = "l1", **adam_kw) -> None:
    """Write a fit's state (efunc_checkpoint_save): params, m, v (CUDA or CPU
    tensors of R^3 * channels floats), the number of Adam steps taken and the
    fit's configuration; efunc_fit(..., step0=step) continues it."""
    n = params.numel()
    if channels < 1 or n % channels:
        raise ValueError("params must hold R^3 * channels floats")
    R = round((n // channels) ** (1.0 / 3.0))
    if R ** 3 * channels != n:
        raise ValueError("params must hold R^3 * channels floats")
    hp, hm, hv = (_host_f32(t, n, nm) for t, nm in ((params, "params"), (m, "m"), (v, "v")))
    info = B.CheckpointInfo(R, W, default_log_beta0(R) if log_beta0 is None else float(log_beta0), channels, n,
                            int(step), int(seed), {"l1": B.LOSS_L1, "mse": B.LOSS_MSE}[loss], make_adam(**adam_kw))
    B.check("efunc_checkpoint_save", B.load().efunc_checkpoint_save(
        str(path).encode(), ctypes.byref(info), _ptr(hp), _ptr(hm), _ptr(hv)))


def load_checkpoint(path: str, device="cuda") -> dict:
    """Read a checkpoint written by save_checkpoint (efunc_checkpoint_load):
    params, m, v on ``device`` and the stored step, seed, loss, grid and Adam
    settings.  A missing, short or corrupt file raises EfuncError
    (EFUNC_ERR_IO)."""
    lib = B.load()
    info = B.CheckpointInfo()
    B.check("efunc_checkpoint_info_read", lib.efunc_checkpoint_info_read(str(path).encode(), ctypes.byref(info)))
    n = int(info.n)
    arrays = [torch.empty(n, dtype=torch.float32) for _ in range(3)]
    B.check("efunc_checkpoint_load", lib.efunc_checkpoint_load(
        str(path).encode(), ctypes.byref(info), *(_ptr(a) for a in arrays), n))
    a = info.adam
    return {"params": arrays[0].to(device), "m": arrays[1].to(device), "v": arrays[2].to(device),
            "step": int(info.step), "seed": int(info.seed), "loss": {B.LOSS_L1: "l1", B.LOSS_MSE: "mse"}[info.loss],
            "R": int(info.R), "W": int(info.W), "log_beta0": float(info.log_beta0), "channels": int(info.channels),
            "adam": {"lr": a.lr, "beta1": a.beta1, "beta2": a.beta2, "eps": a.eps, "weight_decay": a.weight_decay,
                     "decoupled": bool(a.decoupled)}}


def efunc_adam_step(params, grad, m, v, step: int, **adam_kw):
    """One Adam/AdamW step in place; grad is zeroed."""
    for t, nm in ((params, "params"), (grad, "grad"), (m, "m"), (v, "v")):
        _need(t, nm, params.numel())
    ad = make_adam(**adam_kw)
    B.check("efunc_adam_step", B.load().efunc_adam_step(ctypes.byref(ad), params.numel(), _ptr(params), _ptr(grad),
                                                        _ptr(m), _ptr(v), int(step), _stream(params.device)))


def efunc_fit(params, m, v, qo, steps: int, J: int | None = None, n_batches: int = 1, step0: int = 0,
              loss: str = "l1", stats=None, log_beta0: float | None = None, ws: Workspace | None = None,
              eikonal_weight: float = 0.0, pipelined: bool = True, graph: bool = False, **adam_kw):
    """Fitting loop (Sec. 3.4) on batches of (x, y, z, target) rows.

    ``qo`` is a CUDA tensor or a (pinned) CPU tensor of n_batches*J rows of 4
    floats; ``stats`` (optional, CUDA or CPU float32 tensor of steps*2) gets
    (loss, MAE) per step.  ``pipelined`` sizes the workspace for the sort of
    the next batch to run beside the current one (else batches are sorted in
    line).  ``graph`` replays the pipelined schedule from a CUDA graph
    (efunc_fit_graph: device batches and statistics only)."""
    if graph and not pipelined:
        raise ValueError("the graph-replayed fit is the pipelined schedule")
    R = resolution_of(params)
    for t, nm in ((params, "params"), (m, "m"), (v, "v")):
        _need(t, nm, params.numel())
    if qo.dtype != torch.float32 or not qo.is_contiguous() or qo.dim() != 2 or qo.shape[1] != 4:
        raise ValueError("qo must be a contiguous float32 (n_batches*J, 4) tensor")
    if J is None:
        J = qo.shape[0] // n_batches
    if J * n_batches != qo.shape[0]:
        raise ValueError("qo must hold n_batches * J rows")
    if stats is not None and (stats.dtype != torch.float32 or stats.numel() < 2 * steps or not stats.is_contiguous()):
        raise ValueError("stats must be a contiguous float32 tensor of at least 2*steps")
    grid = make_grid(R, log_beta0)
    ad = make_adam(**adam_kw)
    buf, n = _workspace(params.device, ws).get(grid, J, fit=pipelined)
    if not pipelined:
        n = int(B.load().efunc_workspace_bytes(ctypes.byref(grid), int(J)))
    lk = {"l1": B.LOSS_L1, "mse": B.LOSS_MSE}[loss]
    name = "efunc_fit_graph" if graph else "efunc_fit"
    B.check(name, getattr(B.load(), name)(ctypes.byref(grid), ctypes.byref(ad), lk, float(eikonal_weight),
                                          _ptr(params), _ptr(m), _ptr(v),
                                          _ptr(qo), J, n_batches, steps, step0, _ptr(stats), _ptr(buf), n,
                                          _stream(params.device)))


class EfuncFn(torch.autograd.Function):
    """O = EfuncFn.apply(params, q): differentiable in params and q.

    Forward: Algorithm 1.  Backward: Algorithm 2 for dL/dparams and
    Eq. func-normal for dL/dq, both recomputed from (params, q).  float32
    tensors run the hot-path kernels, float64 tensors their FP64
    instantiation (for torch.autograd.gradcheck)."""

    @staticmethod
    def forward(ctx, params, q, log_beta0=None):
        ctx.save_for_backward(params, q)
        ctx.log_beta0 = log_beta0
        fwd = efunc_forward_f64 if params.dtype == torch.float64 else efunc_forward
        return fwd(params.detach().contiguous(), q.detach().contiguous(), log_beta0=log_beta0)

    @staticmethod
    def backward(ctx, gO):
        params, q = ctx.saved_tensors
        need_q = ctx.needs_input_grad[1]
        bwd = efunc_backward_f64 if params.dtype == torch.float64 else efunc_backward
        out = bwd(params.detach().contiguous(), q.detach().contiguous(), gO.contiguous(),
                  want_gq=need_q, log_beta0=ctx.log_beta0)
        gp, gq = (out if need_q else (out, None))
        if gq is not None and q.shape[1] == 4:
            gq = torch.cat([gq, torch.zeros_like(gq[:, :1])], 1)
        return (gp if ctx.needs_input_grad[0] else None), gq, None


# ------------------------------------------------------------ batched fit

class Batch:
    """S shapes fitted together (efunc_fit_batched): ``Rs`` grid
    resolutions, ``Js`` queries per batch of each shape.  Parameters of all
    shapes live in one float32 tensor, shape s at offset 13 sum_{s'<s} R^3;
    a batch is (sum J, 4) rows, the shapes' rows in order."""

    def __init__(self, Rs, Js, log_beta0s=None, device="cuda"):
        if len(Rs) != len(Js) or not Rs:
            raise ValueError("Rs and Js must be non-empty and of equal length")
        lbs = [default_log_beta0(R) for R in Rs] if log_beta0s is None else list(log_beta0s)
        self.S = len(Rs)
        self.Rs, self.Js = [int(r) for r in Rs], [int(j) for j in Js]
        self.shapes = (B.Shape * self.S)(*[B.Shape(int(R), float(lb), int(J)) for R, lb, J in zip(Rs, lbs, Js)])
        lib = B.load()
        self.n_params = int(lib.efunc_batched_param_count(self.shapes, self.S))
        self.n_queries = int(lib.efunc_batched_query_count(self.shapes, self.S))
        if self.n_params < 0 or self.n_queries < 0:
            raise ValueError("invalid shape list")
        self.param_offsets = [0]
        self.query_offsets = [0]
        for R, J in zip(self.Rs, self.Js):
            self.param_offsets.append(self.param_offsets[-1] + 13 * R ** 3)
            self.query_offsets.append(self.query_offsets[-1] + J)
        self.device = torch.device(device)
        self.ws = torch.empty(int(lib.efunc_batched_workspace_bytes(self.shapes, self.S)), dtype=torch.uint8,
                              device=self.device)
        self.tuning = None

    def params_of(self, t: torch.Tensor, s: int) -> torch.Tensor:
        return t[self.param_offsets[s]:self.param_offsets[s + 1]]

    def rows_of(self, batch: torch.Tensor, s: int) -> torch.Tensor:
        return batch[self.query_offsets[s]:self.query_offsets[s + 1]]

    def _tuning(self):
        return ctypes.byref(self.tuning) if self.tuning is not None else None

    def fit(self, params, m, v, qo, steps: int, n_batches: int = 1, step0: int = 0, loss: str = "l1", stats=None,
            graph: bool = True, **adam_kw):
        for t, nm in ((params, "params"), (m, "m"), (v, "v")):
            _need(t, nm, self.n_params)
        _need(qo, "qo", 4 * self.n_queries * n_batches)
        if stats is not None:
            _need(stats, "stats", 2 * self.S * steps)
        ad = make_adam(**adam_kw)
        lk = {"l1": B.LOSS_L1, "mse": B.LOSS_MSE}[loss]
        B.check("efunc_fit_batched", B.load().efunc_fit_batched(
            self.shapes, self.S, ctypes.byref(ad), lk, _ptr(params), _ptr(m), _ptr(v), _ptr(qo), n_batches, steps,
            step0, _ptr(stats), self._tuning(), int(bool(graph)), _ptr(self.ws), self.ws.numel(),
            _stream(self.device)))

    def eval(self, params, qo) -> torch.Tensor:
        """(S, 2): mean squared and mean absolute error of every shape on qo."""
        _need(params, "params", self.n_params)
        _need(qo, "qo", 4 * self.n_queries)
        out = torch.empty((self.S, 2), dtype=torch.float32, device=self.device)
        B.check("efunc_eval_batched", B.load().efunc_eval_batched(
            self.shapes, self.S, _ptr(params), _ptr(qo), _ptr(out), self._tuning(), _ptr(self.ws), self.ws.numel(),
            _stream(self.device)))
        return out

    def tune(self, params, m, v, qo, n_batches: int = 1, trial_steps: int = 3, loss: str = "l1"):
        """Pick the fastest launch configuration (efunc_tune_batched); params
        unchanged, m and v zeroed.  Returns (tuning dict, ms per step)."""
        best = B.Tuning()
        ms = ctypes.c_double(0)
        lk = {"l1": B.LOSS_L1, "mse": B.LOSS_MSE}[loss]
        B.check("efunc_tune_batched", B.load().efunc_tune_batched(
            self.shapes, self.S, lk, _ptr(params), _ptr(m), _ptr(v), _ptr(qo), n_batches, trial_steps,
            ctypes.byref(best), ctypes.byref(ms), _ptr(self.ws), self.ws.numel(), _stream(self.device)))
        self.tuning = best
        return ({"chunk": best.chunk, "lanes2_max": best.lanes2_max, "lanes4_max": best.lanes4_max,
                 "sort_blocks": best.sort_blocks, "group_max": best.group_max}, ms.value)


# ------------------------------------------------------ warm-start encoder

ENC_R = 32


def encoder_weight_count() -> int:
    return int(B.load().efunc_encoder_weight_count())


def encoder_init(seed: int = 0) -> torch.Tensor:
    """He-initialised FP32 master weights of the encoder (CPU tensor; biases 0)."""
    import numpy as np
    g = np.random.Generator(np.random.Philox(int(seed)))
    parts = []
    for fan_in, n_w, n_b in ((27, 32 * 27, 32), (27 * 32, 64 * 27 * 32, 64), (27 * 64, 128 * 27 * 64, 128),
                             (128, 13 * 128, 13)):
        parts.append(g.standard_normal(n_w) * np.sqrt(2.0 / fan_in))
        parts.append(np.zeros(n_b))
    w = np.concatenate(parts).astype(np.float32)
    assert w.size == encoder_weight_count()
    return torch.from_numpy(w)


class Encoder:
    """Workspace-holding wrapper of the encoder calls for a fixed batch size."""

    def __init__(self, batch: int, device="cuda"):
        self.batch = int(batch)
        self.device = torch.device(device)
        n = int(B.load().efunc_encoder_workspace_bytes(self.batch))
        if n == 0:
            raise ValueError("invalid batch")
        self.ws = torch.empty(n, dtype=torch.uint8, device=self.device)

    def forward(self, weights, sdf):
        """(batch, 32^3 x 13) predicted parameter grids from (batch, 32, 32, 32) SDF grids."""
        _need(weights, "weights", encoder_weight_count())
        _need(sdf, "sdf", self.batch * ENC_R ** 3)
        out = torch.empty((self.batch, ENC_R ** 3 * NSLOT), dtype=torch.float32, device=self.device)
        B.check("efunc_encoder_forward", B.load().efunc_encoder_forward(
            _ptr(weights), _ptr(sdf), self.batch, _ptr(out), _ptr(self.ws), self.ws.numel(), _stream(self.device)))
        return out

    def train_step(self, weights, sdf, target, slot_weights=None):
        """(grad, loss): dL/dweights and the weighted MSE of one batch."""
        _need(weights, "weights", encoder_weight_count())
        _need(sdf, "sdf", self.batch * ENC_R ** 3)
        _need(target, "target", self.batch * ENC_R ** 3 * NSLOT)
        if slot_weights is not None:
            _need(slot_weights, "slot_weights", NSLOT)
        grad = torch.empty_like(weights)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        B.check("efunc_encoder_train_step", B.load().efunc_encoder_train_step(
            _ptr(weights), _ptr(sdf), _ptr(target), _ptr(slot_weights), self.batch, _ptr(grad), _ptr(loss),
            _ptr(self.ws), self.ws.numel(), _stream(self.device)))
        return grad, loss

    def status(self):
        B.check("efunc_encoder_status", B.load().efunc_encoder_status(_ptr(self.ws)))


def profile(enable: bool = True):
    B.load().efunc_profile_enable(int(enable))


def profile_read(name: str) -> tuple[float, int]:
    ms, cnt = ctypes.c_double(0), ctypes.c_int64(0)
    rc = B.load().efunc_profile_read(name.encode(), ctypes.byref(ms), ctypes.byref(cnt))
    if rc != 0:
        raise RuntimeError(f"efunc_profile_read({name}) failed")
    return ms.value, cnt.value


def profile_reset():
    B.load().efunc_profile_reset()


def launch_count() -> int:
    return int(B.load().efunc_launch_count())


def debug_bounds() -> int | None:
    """The first bounds-check code the kernels recorded on the current device
    since the last call (0: none), cleared; None unless the bounds-check build
    is loaded (EFUNC_DEBUG_BOUNDS=1)."""
    code = ctypes.c_int32(0)
    st = B.load().efunc_debug_bounds(ctypes.byref(code))
    if st == 5:   # EFUNC_ERR_UNSUPPORTED: the normal build
        return None
    B.check("efunc_debug_bounds", st)
    return int(code.value)
