"""Rounding to the storage formats of Table 1 (test infrastructure).

The paper simulates low-precision work types by rounding (Sec. 2, Table 1).
Here each format is written from its bit layout: a value is rounded to the
nearest representable number, ties to even, straight from binary64 (no
double rounding through binary32).

Table 1 lists, per format, f_max, f_min (smallest normal), f_smin (smallest
subnormal) and machine epsilon; ``FORMAT_LIMITS`` restates those numbers as
they follow from (exponent bits e, mantissa bits m).
"""
from __future__ import annotations

import numpy as np

__all__ = ["FORMATS", "format_limits", "round_real", "round_complex", "machine_eps"]

# name -> (exponent bits, explicit mantissa bits)
FORMATS = {
    "fp64": (11, 52),
    "fp32": (8, 23),
    "fp16": (5, 10),
    "bf16": (8, 7),
    "tf32": (8, 10),
}


def format_limits(name: str) -> dict:
    """f_max, f_min, f_smin and eps of an IEEE-style binary format."""
    e, m = FORMATS[name]
    bias = 2 ** (e - 1) - 1
    emax = bias
    emin = 1 - bias
    return {
        "f_max": (2.0 - 2.0 ** (-m)) * 2.0 ** emax,
        "f_min": 2.0 ** emin,
        "f_smin": 2.0 ** (emin - m),
        "eps": 2.0 ** (-m),
    }


def machine_eps(name: str) -> float:
    return format_limits(name)["eps"]


def round_real(x, name: str) -> np.ndarray:
    """Round binary64 values to format ``name`` (RNE, gradual underflow).

    Values beyond f_max (after rounding) become +-inf, as in IEEE arithmetic.
    """
    x = np.asarray(x, dtype=np.float64)
    if name == "fp64":
        return x.copy()
    e, m = FORMATS[name]
    lim = format_limits(name)
    emin = int(np.log2(lim["f_min"]))
    # exponent of the leading bit (exact, from frexp), clamped at emin so
    # that subnormals share the fixed quantum 2^(emin - m)
    _, ex = np.frexp(x)
    ex = np.maximum(ex.astype(np.float64) - 1.0, emin)
    quantum = np.exp2(ex - m)
    q = np.round(x / quantum) * quantum  # np.round: ties to even
    q = np.where(np.abs(q) > lim["f_max"], np.copysign(np.inf, x), q)
    return q


def round_complex(z, name: str) -> np.ndarray:
    z = np.asarray(z, dtype=np.complex128)
    if name == "fp64":
        return z.copy()
    return round_real(z.real, name) + 1j * round_real(z.imag, name)
