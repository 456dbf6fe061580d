"""Measured parity margins: for every tolerance check of the GPU tests, the
largest error and the ratio error / tolerance.  The record is written as
JSON at the end of the session when EFUNC_PARITY_MARGINS names a file, so
the measured headroom of each bound can be read beside the bound itself."""
import json
import os

import numpy as np

_records = {}
_current = ["(no test)"]


def set_test(nodeid):
    _current[0] = nodeid


def record(what, err, lim):
    err = np.asarray(err, dtype=np.float64)
    lim = np.broadcast_to(np.asarray(lim, dtype=np.float64), err.shape).ravel()
    err = err.ravel()
    if err.size == 0:
        return
    ok = np.isfinite(err)
    if not ok.any():
        return
    ratio = err[ok] / np.maximum(lim[ok], 1e-300)
    key = f"{_current[0]} :: {what}"
    prev = _records.get(key)
    worst = float(ratio.max())
    if prev is None or worst > prev["ratio"]:
        _records[key] = {"ratio": worst, "max_err": float(err[ok].max())}


def dump():
    path = os.environ.get("EFUNC_PARITY_MARGINS")
    if not path or not _records:
        return
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "w") as f:
        json.dump(dict(sorted(_records.items())), f, indent=1)
