"""The FP32 expm1 of the fused kernel (Taylor series through x^8 on
|x| <= 1/2, e^x - 1 elsewhere) against the exact function: the series'
truncation error must sit below FP32 rounding on its branch."""
import math

import numpy as np


def series(x):
    x = np.float32(x)
    c = [np.float32(1.0 / math.factorial(k)) for k in range(1, 9)]
    acc = c[-1]
    for ck in reversed(c[:-1]):
        acc = np.float32(ck + x * acc)
    return np.float32(x * acc)


def test_series_branch_accuracy():
    xs = np.concatenate([np.linspace(-0.5, 0.5, 2001), [1e-30, -1e-30, 1e-7, -1e-7, 1e-3]])
    worst = 0.0
    for x in xs:
        ref = math.expm1(float(np.float32(x)))
        if ref == 0.0:
            assert series(x) == 0.0
            continue
        worst = max(worst, abs(float(series(x)) - ref) / abs(ref))
    assert worst < 4 * 2.0 ** -24, worst  # a few FP32 ulps


def test_exp_branch_has_no_cancellation():
    # for |x| > 1/2, |e^x - 1| >= 0.39 e^x: an FP32 error of a few ulps in e^x
    # stays a few ulps in e^x - 1
    for x in (0.5, -0.5, 1.0, -3.0, 5.0):
        assert abs(math.expm1(x)) >= 0.39 * math.exp(x)
