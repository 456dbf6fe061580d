"""Mutation tests of the oracle's pins.

Each case plants one plausible mistake in a copy of the oracle's C source (a
dropped term, a flipped sign, an off-by-one window, swapped slots, a wrong
Taylor factor, a different reading of a garbled formula), builds it, and
checks that at least one pin of test_oracle_pins.py fails against it.  The
mistakes are planted in the oracle only, on the CPU; the CUDA path is not
involved.  A mutant that no pin catches would mean the pins leave that part
of the oracle unchecked.
"""
import hashlib
import inspect

import pytest

import oracle
import test_oracle_pins as P

# name -> (text in efunc_oracle.c, replacement); the text must occur exactly once
MUTANTS = {
    "offset key placed at the grid key (Delta dropped)": (
        "        k.p[0] += th[0]; k.p[1] += th[1]; k.p[2] += th[2];\n        k.beta = exp(log_beta0 + th[4]);",
        "        k.beta = exp(log_beta0 + th[4]);"),
    "value without its linear term": (
        "*f = k->o + k->d[0] * r[0] + k->d[1] * r[1] + k->d[2] * r[2];",
        "*f = k->o;"),
    "exponent without the scale beta": (
        "*expo = -k->beta * (*d2);",
        "*expo = -(*d2);"),
    "grid key reads the offset key's log-scale": (
        "        k.beta = exp(log_beta0 + th[3]);",
        "        k.beta = exp(log_beta0 + th[4]);"),
    "dO/dbeta with the wrong sign": (
        "double dbeta = gl * (-d2 * (f - O));",
        "double dbeta = gl * (d2 * (f - O));"),
    "dO/dDelta without the -d term": (
        "gr[x] += gl * (-k.d[x] + 2.0 * k.beta * r[x] * (f - O));",
        "gr[x] += gl * (2.0 * k.beta * r[x] * (f - O));"),
    "dO/dq without the 2 beta (q - p)(O - f) term": (
        "g[x] += w * (k.d[x] + 2.0 * k.beta * r[x] * (O - f));",
        "g[x] += w * k.d[x];"),
    "window one centre low": (
        "int l = c - W + 1, h = c + W;",
        "int l = c - W, h = c + W - 1;"),
    "window base without the half-cell shift": (
        "float u = t - 0.5f;",
        "float u = t;"),
    "L1 gradient with sign(0) = 1": (
        "(diff > 0.0 ? 1.0 : (diff < 0.0 ? -1.0 : 0.0))",
        "(diff >= 0.0 ? 1.0 : -1.0)"),
    "Adam without the first-moment bias correction": (
        "double mhat = m[i] / bc1;",
        "double mhat = m[i];"),
    "second order: dG/dd without the + u term": (
        "g_d[x] = w * (r[x] * e1 + u[x]) + go * w * r[x];",
        "g_d[x] = w * (r[x] * e1) + go * w * r[x];"),
    "variant: quadratic term without the 1/2": (
        "v += 0.5 * S[a][b] * x[a] * x[b];",
        "v += S[a][b] * x[a] * x[b];"),
    "variant: cubic term with 1/2 instead of 1/6": (
        "v += T[a][b][c] * x[a] * x[b] * x[c] / 6.0;",
        "v += T[a][b][c] * x[a] * x[b] * x[c] / 2.0;"),
    "variant: offset gradient without grad f": (
        "k.grad_delta[i] += gl * (-g[i] + 2.0 * k.beta * x[i] * (f - O));",
        "k.grad_delta[i] += gl * (2.0 * k.beta * x[i] * (f - O));"),
    "variant: learnable-scale gradient without the chain factor beta": (
        "if (k.grad_b) *k.grad_b += gl * k.beta * (-d2 * (f - O));",
        "if (k.grad_b) *k.grad_b += gl * (-d2 * (f - O));"),
    "mean shift returns the weighted mean, not the offset": (
        "dl[x] = S[x] / Z - k[x];",
        "dl[x] = S[x] / Z;"),
    "cosine weight read as cos(b pi (x + y + z))": (
        "return cos(b * pi * q[0]) * cos(b * pi * q[1]) * cos(b * pi * q[2]);",
        "return cos(b * pi * (q[0] + q[1] + q[2]));"),
    "window upper clamp at R instead of R - 1": (
        "float lo = -1.0f, hi = (float)(R - 1);",
        "float lo = -1.0f, hi = (float)R;"),
    "centres at cell corners": (
        "return -1.0 + ((double)idx + 0.5) * (2.0 / (double)R);",
        "return -1.0 + ((double)idx) * (2.0 / (double)R);"),
    "global brute force over grid keys only": (
        "            for (int s = 0; s < 2; ++s) {\n                key_t_ k = make_key(params, R, log_beta0, a, b, c, s);\n"
        "                double r[3], d2;",
        "            for (int s = 0; s < 1; ++s) {\n                key_t_ k = make_key(params, R, log_beta0, a, b, c, s);\n"
        "                double r[3], d2;"),
    "second order: T without its factor -2": (
        "const double T = -2.0 * (u[0] * V[0] + u[1] * V[1] + u[2] * V[2]);",
        "const double T = (u[0] * V[0] + u[1] * V[1] + u[2] * V[2]);"),
    "second order: dG/dbeta without the -2 dlt u.r term": (
        "const double g_beta = w * (-d2 * hH - 2.0 * dlt * ur) + go * w * (-d2 * dlt);",
        "const double g_beta = w * (-d2 * hH) + go * w * (-d2 * dlt);"),
    "second order: dG/dDelta without 2 beta dlt u": (
        "g_p[x] = w * (2.0 * k.beta * r[x] * hH - k.d[x] * e1 + 2.0 * k.beta * dlt * u[x]) +",
        "g_p[x] = w * (2.0 * k.beta * r[x] * hH - k.d[x] * e1) +"),
    "mean shift without the largest-exponent shift": (
        "const double w = exp(-bw * d2 - M);",
        "const double w = exp(-bw * d2);"),
    "variant: quadratic gradient with a 1/2": (
        "g[a] += S[a][b] * x[b];",
        "g[a] += 0.5 * S[a][b] * x[b];"),
    "variant: cubic gradient with 1/6 instead of 1/2": (
        "g[a] += 0.5 * T[a][b][c] * x[b] * x[c];",
        "g[a] += T[a][b][c] * x[b] * x[c] / 6.0;"),
    "variant: S_xy stored on one side only": (
        "S[0][1] = S[1][0] = phi[7];",
        "S[0][1] = phi[7];"),
    "cosine backward without the band weight": (
        "variant_one(params + b * band, grad + b * band, gS[j] * cosine_weight(b, qj), R, W, log_beta0, 1, 1, 1,",
        "variant_one(params + b * band, grad + b * band, gS[j], R, W, log_beta0, 1, 1, 1,"),
    "cosine bands counted from 1": (
        "s += cosine_weight(b, qj) * O;",
        "s += cosine_weight(b + 1, qj) * O;"),
    "MSE gradient without the factor 2": (
        "gO[j] = 2.0 * diff / (double)J;",
        "gO[j] = diff / (double)J;"),
    "AdamW decay and Adam L2 penalty swapped": (
        "        if (decoupled)\n            p[i] *= 1.0 - lr * wd;",
        "        if (!decoupled)\n            p[i] *= 1.0 - lr * wd;"),
    "Adam eps inside the square root": (
        "p[i] -= lr * mhat / (sqrt(vhat) + eps);",
        "p[i] -= lr * mhat / sqrt(vhat + eps);"),
    "tolerance diagnostic: kappa without the weights' own rounding": (
        "k_sum += exp(expo - M) / e * (fabs(expo) + 1.0) * fabs(f - O);",
        "k_sum += exp(expo - M) / e * fabs(expo) * fabs(f - O);"),
    "tolerance diagnostic: dO/dq sensitivity without its factor 2": (
        "*dq_sens = 2.0 * sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);",
        "*dq_sens = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);"),
    "tolerance diagnostic: kappa_G without the weights' own rounding": (
        "k_sum += w * (fabs(expo) + 1.0) * sqrt(dev2);",
        "k_sum += w * fabs(expo) * sqrt(dev2);"),
    "tolerance diagnostic: dO/dq's fabs without the constant term": (
        "fa += w * (fabs(k.o) + fabs(k.d[0] * r[0]) + fabs(k.d[1] * r[1]) + fabs(k.d[2] * r[2]));",
        "fa += w * (fabs(k.d[0] * r[0]) + fabs(k.d[1] * r[1]) + fabs(k.d[2] * r[2]));"),
    "tolerance diagnostic: gabs without |O - f|": (
        "const double ax = fabs(k.d[x]) + 2.0 * k.beta * fabs(r[x]) * fabs(O - f);",
        "const double ax = fabs(k.d[x]) + 2.0 * k.beta * fabs(r[x]);"),
    "tolerance diagnostic: kappa_G with the key term's 2 dropped": (
        "const double gx = k.d[x] + 2.0 * k.beta * r[x] * (O - f) - G[x];",
        "const double gx = k.d[x] + k.beta * r[x] * (O - f) - G[x];"),
    "tolerance diagnostic: gradient error terms without |f - O| in the Delta term": (
        "t[x] = gl * (fabs(k.d[x]) + 2.0 * k.beta * fabs(r[x]) * fabs(f - O));",
        "t[x] = gl * (fabs(k.d[x]) + 2.0 * k.beta * fabs(r[x]));"),
    "tolerance diagnostic: gradient error terms weighted by |exponent| only": (
        "const double we = fabs(expo) + 1.0;",
        "const double we = fabs(expo);"),
    "tolerance diagnostic: variant fabs as |f| instead of its terms": (
        "fa += fabs(k.phi[i] * fu);",
        "fa += k.phi[i] * fu;"),
}


def pin_cases():
    """Every pin of test_oracle_pins.py with its parametrisations expanded."""
    for name, fn in sorted(inspect.getmembers(P, inspect.isfunction)):
        if not name.startswith("test_"):
            continue
        combos = [{}]
        for mark in getattr(fn, "pytestmark", []):
            if mark.name != "parametrize":
                continue
            names = [n.strip() for n in mark.args[0].split(",")]
            expanded = []
            for c in combos:
                for vals in mark.args[1]:
                    vals = vals if len(names) > 1 else (vals,)
                    d = dict(c)
                    d.update(zip(names, vals))
                    expanded.append(d)
            combos = expanded
        if set(inspect.signature(fn).parameters) - set(combos[0]):
            continue   # needs a fixture: not a pure pin
        for c in combos:
            yield name, fn, c


def first_failing_pin(path):
    with oracle.swapped_library(path):
        for name, fn, kw in pin_cases():
            try:
                fn(**kw)
            except Exception:   # an assertion or an error: the pin suite fails
                return name
    return None


def test_pins_pass_on_the_unmodified_source():
    text = oracle.source_text()
    path = oracle.build_variant_source(text, "unmodified_copy")
    assert first_failing_pin(path) is None


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_pins_catch_planted_mistake(mutant):
    old, new = MUTANTS[mutant]
    text = oracle.source_text()
    assert text.count(old) == 1, f"mutation target not unique or missing: {old!r}"
    tag = hashlib.sha1(mutant.encode()).hexdigest()[:10]
    path = oracle.build_variant_source(text.replace(old, new), "mutant_" + tag)
    caught = first_failing_pin(path)
    assert caught is not None, f"no pin fails with the mistake: {mutant}"
