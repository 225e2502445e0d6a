"""Host checks of the synthetic-array support of the CUDA path (no GPU):
the double-float sine/cosine table compiled into the kernels, and the
uniform-linear-array layout the binding hands over."""
import math
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ARRAY_CUH = os.path.join(ROOT, "paper_2504_21719_b300", "csrc", "array.cuh")


def _table():
    src = open(ARRAY_CUH).read()
    body = src[src.index("SINCOS_PI_64[65][4] = {"):]
    body = body[:body.index("};")]
    rows = re.findall(r"\{([^{}]+)\}", body)
    return np.array([[float(v.strip().rstrip("f")) for v in r.split(",")] for r in rows])


def test_sincos_table_is_sin_and_cos_of_pi_j_over_64():
    """Each row j holds sin(pi j/64) and cos(pi j/64) as hi + lo FP32 pairs:
    hi is the float nearest the value and hi + lo is within 2^-48 of it."""
    t = _table()
    assert t.shape == (65, 4)
    for j in range(65):
        s, c = math.sin(math.pi * j / 64), math.cos(math.pi * j / 64)
        exact = {0: (0.0, 1.0), 32: (1.0, 0.0), 64: (0.0, -1.0)}
        if j in exact:  # the exact values, not libm's rounding of pi j / 64
            s, c = exact[j]
        for col, v in ((0, s), (2, c)):
            hi, lo = t[j, col], t[j, col + 1]
            assert hi == float(np.float32(v)), (j, col)
            assert float(np.float32(lo)) == lo
            assert abs(hi + lo - v) <= 2.0 ** -48 + 1e-16, (j, col, hi + lo - v)
