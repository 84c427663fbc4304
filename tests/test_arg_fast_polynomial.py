"""The polynomial arctangent of the sweep kernel (arg_fast in
csrc/llr_device.cuh), evaluated on the host in float32 arithmetic with the
coefficients read from the header, against numpy's FP64 arctan2: its error
stays below the bound its comment states, in every octant, on the axes and at
zero.  (The GPU evaluation itself is covered by the link-by-link parity of the
overrelaxation and heat-bath passes.)"""
import os
import re

import numpy as np

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_1509_08391_gb300", "csrc",
                   "llr_device.cuh")


def _coefficients():
    src = open(HDR).read()
    body = src[src.index("float arg_fast("):]
    body = body[:body.index("return copysignf")]
    first = re.search(r"float p = (-?[0-9.]+)f;", body).group(1)
    rest = re.findall(r"p = fmaf\(p, u, (-?[0-9.]+)f\);", body)
    return [np.float32(first)] + [np.float32(c) for c in rest]


def _fma32(a, b, c):
    # a * b is exact in float64 for float32 inputs; one rounding to float32
    # of the float64 sum differs from a true fma only in double-rounding ties
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def _arg_fast(y, x):
    y = y.astype(np.float32)
    x = x.astype(np.float32)
    ax, ay = np.abs(x), np.abs(y)
    mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
    t = (mn / np.maximum(mx, np.float32(1e-30))).astype(np.float32)
    u = (t * t).astype(np.float32)
    c = _coefficients()
    p = np.full_like(u, c[0])
    for cj in c[1:]:
        p = _fma32(p, u, np.full_like(u, cj))
    r = (t * p).astype(np.float32)
    r = np.where(ay > ax, (np.float32(np.pi / 2) - r).astype(np.float32), r)
    r = np.where(x < 0, (np.float32(np.pi) - r).astype(np.float32), r)
    return np.copysign(r, y)


def test_polynomial_has_eight_coefficients():
    assert len(_coefficients()) == 8


def test_error_bound_over_all_octants():
    phi = np.linspace(-np.pi, np.pi, 400_001)
    for rad in (1e-3, 0.7, 3.0, 6.0):
        y = (rad * np.sin(phi)).astype(np.float32)
        x = (rad * np.cos(phi)).astype(np.float32)
        got = _arg_fast(y, x).astype(np.float64)
        ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
        d = np.angle(np.exp(1j * (got - ref)))          # modulo 2 pi (at +-pi)
        # 1.4e-7 polynomial + 1.2e-7 quotient + half an ulp of pi
        assert np.max(np.abs(d)) < 4e-7, rad


def test_axes_and_zero():
    y = np.array([0.0, 1.0, 0.0, -1.0, 0.0, -0.0], dtype=np.float32)
    x = np.array([1.0, 0.0, -1.0, 0.0, 0.0, -1.0], dtype=np.float32)
    got = _arg_fast(y, x)
    ref = np.array([0.0, np.pi / 2, np.pi, -np.pi / 2, 0.0, -np.pi])
    assert np.allclose(got, ref, rtol=0, atol=3e-7)
