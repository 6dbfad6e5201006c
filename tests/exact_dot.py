"""Correctly rounded complex inner products of binary64 data (test reference).

<v, w> = sum_p conj(v_p) w_p, real part sum (vr wr + vi wi), imaginary part
sum (vr wi - vi wr).  Every binary64 product x y is written exactly as four binary64
terms by Veltkamp's splitting of each factor into two halves of at most 26 significant
bits (Dekker 1971: the four partial products of the halves are exact), and math.fsum
returns the correctly rounded sum of all terms (Shewchuk's exact partials).  Valid
while no factor exceeds about 2^995 in magnitude (the splitting constant 2^27 + 1 must
not overflow) and no partial product underflows, which the test inputs respect.
"""
import math

import numpy as np

_SPLIT = float(2 ** 27 + 1)


def split(x):
    """x = hi + lo exactly, hi and lo with at most 26 significant bits each."""
    x = np.asarray(x, dtype=np.float64)
    c = _SPLIT * x
    hi = c - (c - x)
    return hi, x - hi


def product_terms(x, y):
    """Four arrays whose elementwise sum is x * y exactly."""
    xh, xl = split(x)
    yh, yl = split(y)
    return [xh * yh, xh * yl, xl * yh, xl * yl]


def exact_dot(v, w):
    """The correctly rounded <v, w> of two complex128 vectors."""
    v = np.asarray(v, dtype=np.complex128).ravel()
    w = np.asarray(w, dtype=np.complex128).ravel()
    vr, vi, wr, wi = v.real, v.imag, w.real, w.imag
    re = product_terms(vr, wr) + product_terms(vi, wi)
    im = product_terms(vr, wi) + [-t for t in product_terms(vi, wr)]
    re_sum = math.fsum(np.concatenate(re).tolist())
    im_sum = math.fsum(np.concatenate(im).tolist())
    return complex(re_sum, im_sum)
