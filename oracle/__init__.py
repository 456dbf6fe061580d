"""FP64 CPU oracle for the efunc O^{+Delta} representation (arXiv 2505.21319).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product path (the
CUDA library and its Python binding) never imports this package.

The arithmetic lives in ``efunc_oracle.c`` (plain C, FP64, single thread),
which this module compiles with gcc on first use and wraps with ctypes.  Every
function states the passage of the paper it follows; see the C file's header
for the readings it fixes (domain, slot order, log-scale storage, window).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "efunc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libefunc_oracle.so")
_lock = threading.Lock()
_lib = None

NSLOT = 13
L1, MSE = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libefunc_oracle.so``.

    ``-ffp-contract=off`` keeps the FP32 window decision free of fused
    multiply-adds on every host (aarch64 gcc contracts by default)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _configure(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.ora_window_base.argtypes = [ctypes.c_float, i32]
    lib.ora_window_base.restype = i32
    lib.ora_forward.argtypes = [i32, i32, f64, dp, dp, i64, i32, dp, dp, dp, dp, dp]
    lib.ora_backward.argtypes = [i32, i32, f64, dp, dp, i64, i32, dp, dp, dp]
    lib.ora_forward_err_terms.argtypes = [i32, i32, f64, dp, dp, i64, i32, dp, dp, dp]
    lib.ora_backward_err_terms.argtypes = [i32, i32, f64, dp, dp, i64, i32, dp, dp, dp]
    lib.ora_forward_global.argtypes = [i32, f64, dp, dp, i64, i32, dp, dp]
    lib.ora_backward_grad.argtypes = [i32, i32, f64, dp, dp, i64, i32, dp, dp, dp]
    lib.ora_mean_shift.argtypes = [i32, f64, dp, i64, dp]
    lib.ora_variant_channels.argtypes = [i32, i32, i32]
    lib.ora_variant_channels.restype = i32
    lib.ora_variant_forward.argtypes = [i32, i32, f64, i32, i32, i32, dp, dp, i64, i32, dp, dp, dp, dp]
    lib.ora_variant_backward.argtypes = [i32, i32, f64, i32, i32, i32, dp, dp, i64, i32, dp, dp]
    lib.ora_cosine_forward.argtypes = [i32, i32, f64, i32, dp, dp, i64, i32, dp]
    lib.ora_cosine_backward.argtypes = [i32, i32, f64, i32, dp, dp, i64, i32, dp, dp]
    lib.ora_loss_grad.argtypes = [i32, dp, dp, i64, dp, dp, dp]
    lib.ora_adam.argtypes = [i64, dp, dp, dp, dp, i64, f64, f64, f64, f64, f64, i32]
    for fn in ("ora_forward", "ora_forward_err_terms", "ora_backward_err_terms", "ora_backward", "ora_forward_global", "ora_loss_grad", "ora_adam",
               "ora_backward_grad", "ora_mean_shift", "ora_variant_forward", "ora_variant_backward",
               "ora_cosine_forward", "ora_cosine_backward"):
        getattr(lib, fn).restype = None
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _configure(ctypes.CDLL(_LIB_PATH))
    return _lib


def build_variant_source(text: str, name: str) -> str:
    """Compile a modified copy of the oracle's C source (mutation tests of
    the pins) into ``oracle/_build/<name>.so``; returns its path."""
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_BUILD, name + ".c")
    out = os.path.join(_BUILD, name + ".so")
    with open(src, "w") as f:
        f.write(text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                    "-o", out, src, "-lm"], check=True)
    return out


class swapped_library:
    """Context manager: every oracle function uses the library at ``path``
    (a build of a modified source) until the block exits."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _lib
        self.saved = _load()
        _lib = _configure(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def default_log_beta0(R: int) -> float:
    """log(beta) at initialisation.  Sec. 4.3 initialises every scale to exp(7)
    (stated for the 32^3 grid); keeping beta*h^2 fixed across resolutions gives
    7 + 2 ln(R/32)."""
    return 7.0 + 2.0 * float(np.log(R / 32.0))


def window_base(q: float, R: int) -> int:
    """FP32 window base index along one axis (C function ``ora_window_base``)."""
    return int(_load().ora_window_base(ctypes.c_float(float(np.float32(q))), R))


def _check(params, q, R):
    params = _f64(params).reshape(-1)
    if params.size != R ** 3 * NSLOT:
        raise ValueError(f"params must hold R^3*13 = {R**3*NSLOT} values, got {params.size}")
    q = _f64(q)
    if q.ndim != 2 or q.shape[1] < 3:
        raise ValueError("q must be (J, >=3)")
    return params, q


def forward(params, q, R: int, W: int = 2, log_beta0: float | None = None, want_dq: bool = False,
            want_kappa: bool = False, want_dq_sens: bool = False):
    """O(q_j), lse_j (and dO/dq_j, and kappa_j) for the windowed O^{+Delta} model.

    Sec. 3.3 Eq. func-offset evaluated by Algorithm 1 (Sec. 3.5) with the
    log-sum-exp shift; dO/dq from Eq. func-normal.  ``q`` is (J, >=3); only the
    first three columns are read.  W >= R is the paper's global support.
    kappa_j = sum softmax (|exponent| + 1) |f - O| is the condition number of
    O_j with respect to relative rounding of the exponents and the weights (a
    diagnostic used to derive floating-point tolerances).  dq_sens_j =
    2 ||sum softmax beta (q - key)|| is the factor by which an error in O_j
    enters dO/dq_j."""
    lb = default_log_beta0(R) if log_beta0 is None else float(log_beta0)
    params, q = _check(params, q, R)
    J = q.shape[0]
    O = np.zeros(J)
    lse = np.zeros(J)
    dq = np.zeros((J, 3)) if want_dq else None
    kappa = np.zeros(J) if want_kappa else None
    sens = np.zeros(J) if want_dq_sens else None
    _load().ora_forward(R, W, lb, _ptr(params), _ptr(q), J, q.shape[1], _ptr(O), _ptr(lse), _ptr(dq), _ptr(kappa),
                        _ptr(sens))
    out = [O, lse]
    if want_dq:
        out.append(dq)
    if want_kappa:
        out.append(kappa)
    if want_dq_sens:
        out.append(sens)
    return tuple(out)


def dq_error_terms(params, q, R: int, W: int = 2, log_beta0: float | None = None):
    """(kappa_G, fabs, gabs) per query, the error terms of G = dO/dq (Eq.
    func-normal) under relative rounding, with g = d + 2 beta (q - key)(O - f)
    a key's term of G:
      kappa_G = sum softmax (|exponent| + 1) ||g - G||  (rounding of the weights)
      fabs    = sum softmax (|o| + sum_a |d_a r_a|)      (rounding of the values f)
      gabs    = sum softmax ||(|d_a| + 2 beta |r_a| |O - f|)_a||  (of G's terms)
    Diagnostics used to derive the FP32 tolerance of dO/dq."""
    lb = default_log_beta0(R) if log_beta0 is None else float(log_beta0)
    params, q = _check(params, q, R)
    out = [np.zeros(q.shape[0]) for _ in range(3)]
    _load().ora_forward_err_terms(R, W, lb, _ptr(params), _ptr(q), q.shape[0], q.shape[1], *(_ptr(a) for a in out))
    return tuple(out)


def backward(params, q, gO, R: int, W: int = 2, log_beta0: float | None = None, want_gq: bool = False):
    """dL/dtheta (R^3, 13) and optionally dL/dq (J, 3) for upstream dL/dO = gO.

    Algorithm 2 (Sec. 3.6) with the closed-form dO/dk, dO/dbeta, dO/dphi;
    chain rule to the stored log-scale b and to the offset Delta."""
    lb = default_log_beta0(R) if log_beta0 is None else float(log_beta0)
    params, q = _check(params, q, R)
    J = q.shape[0]
    gO = _f64(gO).reshape(-1)
    if gO.size != J:
        raise ValueError("gO must have J entries")
    grad = np.zeros(R ** 3 * NSLOT)
    gq = np.zeros((J, 3)) if want_gq else None
    _load().ora_backward(R, W, lb, _ptr(params), _ptr(q), J, q.shape[1], _ptr(gO), _ptr(grad), _ptr(gq))
    grad = grad.reshape(R ** 3, NSLOT)
    return (grad, gq) if want_gq else grad


def backward_error_terms(params, q, gO, R: int, W: int = 2, log_beta0: float | None = None):
    """(abs0, abs1), (R^3, 13) each: per gradient entry of Algorithm 2 the sum
    of its terms' magnitudes, and the same weighted by (|exponent| + 1) of
    each term's key (the relative error of its weight).  A gradient entry
    whose terms cancel is rounded in proportion to these, not to its value:
    diagnostics for the FP32 tolerance of the gradients."""
    lb = default_log_beta0(R) if log_beta0 is None else float(log_beta0)
    params, q = _check(params, q, R)
    gO = _f64(gO).reshape(-1)
    if gO.size != q.shape[0]:
        raise ValueError("gO must have J entries")
    a0, a1 = np.zeros(R ** 3 * NSLOT), np.zeros(R ** 3 * NSLOT)
    _load().ora_backward_err_terms(R, W, lb, _ptr(params), _ptr(q), q.shape[0], q.shape[1], _ptr(gO), _ptr(a0),
                                   _ptr(a1))
    return a0.reshape(R ** 3, NSLOT), a1.reshape(R ** 3, NSLOT)


def backward_grad(params, q, gO, gG, R: int, W: int = 2, log_beta0: float | None = None):
    """dL/dtheta (R^3, 13) for L = sum_j gO_j O(q_j) + gG_j . dO/dq(q_j).

    The backward through Eq. func-normal (Sec. 3.2) that a loss on the query
    gradient needs (the Eikonal condition |dO/dq|^2 = 1); gO or gG may be None."""
    lb = default_log_beta0(R) if log_beta0 is None else float(log_beta0)
    params, q = _check(params, q, R)
    J = q.shape[0]
    go = None if gO is None else _f64(gO).reshape(-1)
    gg = None if gG is None else _f64(gG).reshape(J, 3)
    grad = np.zeros(R ** 3 * NSLOT)
    _load().ora_backward_grad(R, W, lb, _ptr(params), _ptr(q), J, q.shape[1], _ptr(go), _ptr(gg), _ptr(grad))
    return grad.reshape(R ** 3, NSLOT)


def eikonal_loss_grad(G, weight: float = 1.0):
    """Eikonal term of Sec. 3.2 in the paper's squared form: weight * mean_j
    (|G_j|^2 - 1)^2 and its gradient with respect to G (J, 3)."""
    G = _f64(G).reshape(-1, 3)
    J = G.shape[0]
    res = (G ** 2).sum(1) - 1.0
    loss = weight * float((res ** 2).mean()) if J else 0.0
    gG = weight * 4.0 * res[:, None] * G / J
    return loss, gG


def mean_shift(pts, R: int, bandwidth: float = 100.0):
    """Mean-shift offset initialisation of Sec. 3.3: (R^3, 3) offsets Delta_i =
    softmax-weighted mean of the surface points (weights exp(-bw |k_i - s|^2))
    minus the centre k_i."""
    pts = _f64(pts).reshape(-1, 3)
    delta = np.zeros((R ** 3, 3))
    _load().ora_mean_shift(R, float(bandwidth), _ptr(pts), pts.shape[0], _ptr(delta))
    return delta


def variant_channels(sets: int, deg: int, learn: int) -> int:
    """Floats per centre of an ablation variant (Table tab:ablation "Ch");
    -1 for an invalid description.  sets: 1 grid keys, 2 offset keys, 3 both;
    deg: value polynomial degree 0..3; learn: 1 learnable scales."""
    return int(_load().ora_variant_channels(int(sets), int(deg), int(learn)))


def _variant_check(params, q, R, sets, deg, learn):
    ch = variant_channels(sets, deg, learn)
    if ch < 0:
        raise ValueError("invalid variant")
    params = _f64(params).reshape(R ** 3, ch)
    q = _f64(q)
    if q.ndim != 2 or q.shape[1] not in (3, 4):
        raise ValueError("q must be (J, 3) or (J, 4)")
    return params, q, ch


def variant_forward(params, q, R: int, sets: int, deg: int, learn: int, W: int = 2,
                    log_beta0: float | None = None, want_diag: bool = False):
    """(O, lse) of an ablation variant (Table tab:ablation) at the queries;
    with want_diag also (kappa, fabs): the condition number of O under
    relative rounding of exponents and weights, and sum softmax * sum |terms
    of f| (the scale of f's own rounding)."""
    lb = default_log_beta0(R) if log_beta0 is None else float(log_beta0)
    params, q, _ = _variant_check(params, q, R, sets, deg, learn)
    J = q.shape[0]
    O, lse = np.zeros(J), np.zeros(J)
    kap, fab = (np.zeros(J), np.zeros(J)) if want_diag else (None, None)
    _load().ora_variant_forward(R, W, lb, sets, deg, learn, _ptr(params), _ptr(q), J, q.shape[1], _ptr(O),
                                _ptr(lse), _ptr(kap), _ptr(fab))
    return (O, lse, kap, fab) if want_diag else (O, lse)


def variant_backward(params, q, gO, R: int, sets: int, deg: int, learn: int, W: int = 2,
                     log_beta0: float | None = None):
    """sum_j gO_j dO_j/dparams of an ablation variant, (R^3, channels)."""
    lb = default_log_beta0(R) if log_beta0 is None else float(log_beta0)
    params, q, ch = _variant_check(params, q, R, sets, deg, learn)
    gO = _f64(gO).reshape(-1)
    if gO.shape[0] != q.shape[0]:
        raise ValueError("gO must have one entry per query")
    grad = np.zeros((R ** 3, ch))
    _load().ora_variant_backward(R, W, lb, sets, deg, learn, _ptr(params), _ptr(q), q.shape[0], q.shape[1],
                                 _ptr(gO), _ptr(grad))
    return grad


def _cosine_check(params, q, R, B):
    params = _f64(params).reshape(B, R ** 3, 5)
    q = _f64(q)
    if q.ndim != 2 or q.shape[1] not in (3, 4):
        raise ValueError("q must be (J, 3) or (J, 4)")
    return params, q


def cosine_forward(params, q, R: int, B: int, W: int = 2, log_beta0: float | None = None):
    """S(q) of the cosine-series decomposition (Sec. 4.4): B bands of
    Config-G-6 grids (B x R^3 x 5), weights cos(b pi q_x) cos(b pi q_y) cos(b pi q_z)."""
    lb = default_log_beta0(R) if log_beta0 is None else float(log_beta0)
    params, q = _cosine_check(params, q, R, B)
    S = np.zeros(q.shape[0])
    _load().ora_cosine_forward(R, W, lb, B, _ptr(params), _ptr(q), q.shape[0], q.shape[1], _ptr(S))
    return S


def cosine_backward(params, q, gS, R: int, B: int, W: int = 2, log_beta0: float | None = None):
    """sum_j gS_j dS_j/dparams, (B, R^3, 5)."""
    lb = default_log_beta0(R) if log_beta0 is None else float(log_beta0)
    params, q = _cosine_check(params, q, R, B)
    gS = _f64(gS).reshape(-1)
    grad = np.zeros((B, R ** 3, 5))
    _load().ora_cosine_backward(R, W, lb, B, _ptr(params), _ptr(q), q.shape[0], q.shape[1], _ptr(gS), _ptr(grad))
    return grad


def forward_global(params, q, R: int, log_beta0: float | None = None):
    """Brute force: the paper's global model over all 2I keys (no window)."""
    lb = default_log_beta0(R) if log_beta0 is None else float(log_beta0)
    params, q = _check(params, q, R)
    J = q.shape[0]
    O = np.zeros(J)
    scratch = np.zeros(4 * R ** 3)
    _load().ora_forward_global(R, lb, _ptr(params), _ptr(q), J, q.shape[1], _ptr(O), _ptr(scratch))
    return O


def loss_grad(O, target, loss: int = L1):
    """Upstream gradient dL/dO_j, loss value and mean absolute error.

    Eq. loss (Sec. 3.4) for MSE; L1 = mean |O - o| with sign(0) = 0."""
    O = _f64(O).reshape(-1)
    target = _f64(target).reshape(-1)
    J = O.size
    gO = np.zeros(J)
    L = ctypes.c_double(0.0)
    mae = ctypes.c_double(0.0)
    _load().ora_loss_grad(int(loss), _ptr(O), _ptr(target), J, _ptr(gO), ctypes.byref(L), ctypes.byref(mae))
    return gO, L.value, mae.value


def adam(p, g, m, v, step: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
         eps: float = 1e-8, weight_decay: float = 0.0, decoupled: bool = False):
    """One Adam (or AdamW, ``decoupled=True``) step, torch.optim semantics,
    Sec. 3.4 / Sec. 4.2.  Returns new (p, m, v) as FP64 copies."""
    p = _f64(p).reshape(-1).copy()
    g = _f64(g).reshape(-1)
    m = _f64(m).reshape(-1).copy()
    v = _f64(v).reshape(-1).copy()
    _load().ora_adam(p.size, _ptr(p), _ptr(g), _ptr(m), _ptr(v), int(step), lr, beta1, beta2, eps,
                     weight_decay, int(bool(decoupled)))
    return p, m, v


def fit_step(params, m, v, step: int, qo, R: int, loss: int = L1, lr: float = 1e-3, W: int = 2,
             log_beta0: float | None = None, **adam_kw):
    """One fitting iteration (Sec. 3.4): forward, loss gradient, backward,
    Adam.  ``qo`` is (J, 4) with the target SDF in column 3.  Returns
    (params, m, v, loss, mae) as FP64 arrays / floats."""
    qo = _f64(qo)
    O, _ = forward(params, qo, R, W, log_beta0)
    gO, L, mae = loss_grad(O, qo[:, 3], loss)
    grad = backward(params, qo, gO, R, W, log_beta0)
    p, m, v = adam(params, grad, m, v, step, lr=lr, **adam_kw)
    return p.reshape(-1, NSLOT), m.reshape(-1, NSLOT), v.reshape(-1, NSLOT), L, mae
