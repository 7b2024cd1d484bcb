"""CPU checks of constants the CUDA kernels carry: the polynomials fitted to
p(u) = e2(u)/u^3 that replace the Taylor sums of the interval functions in
the formal solutions without Lambda* (FP32, FP64 and float-float), read from
the kernel sources and compared with the exact function (mpmath).

e2(u) = u^2 - 2 e1(u), e1 = u - (1 - exp(-u)): p(u) = 2 sum_m (-1)^m u^m / (m+3)!.
"""
import os
import re

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2102_01734_gb300", "csrc")
NUM = r"(-?\d+\.\d*(?:e-?\d+)?)f?"


def _function_body(path, signature):
    src = open(os.path.join(CSRC, path)).read()
    i = src.index(signature)
    j = src.index("\n}\n", i)
    return src[i:j]


def _p_exact(u):
    # u^2 - 2 e1 cancels to O(u^3): 60 digits leave 30 after the cancellation
    # for every u >= 1e-10 used here
    with mpmath.workdps(60):
        u = mpmath.mpf(u)
        if u == 0:
            return mpmath.mpf(1) / 3
        e0 = -mpmath.expm1(-u)
        e1 = u - e0
        return (u * u - 2 * e1) / u ** 3


def _horner(coefs, u):
    p = coefs[0]
    for c in coefs[1:]:
        p = p * u + c
    return p


def _nodes(hi, n=400):
    k = np.arange(n)
    return 0.5 * hi * (1 - np.cos(np.pi * (k + 0.5) / n))


def test_fp32_fit_on_unit_interval():
    body = _function_body("fs_step.cuh", "IntervalE interval_fast(")
    coefs = [float(x) for x in re.findall(r"(?:float p =|fmaf\(p, u,) " + NUM, body)]
    assert len(coefs) == 6  # degree 5
    c32 = [np.float32(c) for c in coefs]
    worst_fit = worst_f32 = 0.0
    for u in _nodes(1.0):
        exact = _p_exact(u)
        fit = _horner([mpmath.mpf(float(c)) for c in c32], mpmath.mpf(u))
        worst_fit = max(worst_fit, float(abs(fit / exact - 1)))
        uf = np.float32(u)
        p = c32[0]
        for c in c32[1:]:
            p = np.float32(np.float32(p * uf) + c)
        worst_f32 = max(worst_f32, float(abs(mpmath.mpf(float(p)) / exact - 1)))
    assert worst_fit < 1.0e-7   # the fit itself
    assert worst_f32 < 3.0e-7   # evaluated in FP32 (Horner rounding on top)


def test_fp64_fit_on_half_interval():
    body = _function_body("fs64_step.cuh", "__device__ __forceinline__ IntervalDE interval64(")
    coefs = [float(x) for x in re.findall(r"(?:double p =|fma\(p, u,) " + NUM, body)]
    assert len(coefs) == 10  # degree 9
    worst = 0.0
    with mpmath.workdps(40):
        for u in _nodes(0.5):
            fit = _horner([mpmath.mpf(c) for c in coefs], mpmath.mpf(float(u)))
            worst = max(worst, float(abs(fit / _p_exact(float(u)) - 1)))
    assert worst < 2.0e-16


def test_float_float_fit_on_half_interval():
    body = _function_body("fsff.cu", "IntervalFF interval_ff(")
    high = [float(x) for x in re.findall(r"(?:float q =|fmaf\(q, u\.hi,) " + NUM, body)]
    pairs = re.findall(r"ff\{" + NUM + r", " + NUM + r"\}", body)
    assert len(high) == 4 and len(pairs) == 6  # degree 9: levels 9..6 FP32, 5..0 pairs
    with mpmath.workdps(40):
        coefs = [mpmath.mpf(float(np.float32(c))) for c in high]
        coefs += [mpmath.mpf(float(np.float32(h))) + mpmath.mpf(float(np.float32(l)))
                  for h, l in pairs]
        worst = 0.0
        for u in _nodes(0.5):
            fit = _horner(coefs, mpmath.mpf(float(u)))
            worst = max(worst, float(abs(fit / _p_exact(float(u)) - 1)))
    # levels 9..6 are FP32 numbers: the rounding of c6 (5.5e-6, contributing
    # 8.6e-8 of p at u = 1/2) to 24 bits dominates, about 1e-14 relative; far
    # below the float-float formal solution's per-step error budget (2e-12)
    assert worst < 1.5e-14


def _constexpr_floats(path):
    src = open(os.path.join(CSRC, path)).read()
    return {k: np.float32(float(v)) for k, v in
            re.findall(r"\b(k[A-Z]\w*) = " + NUM, src)}


def _significant_bits(x):
    m, _ = np.frexp(np.float64(x))  # exact for an FP32 value
    m = abs(int(np.ldexp(m, 24)))
    return 24 - (len(bin(m)) - len(bin(m).rstrip("0")))


def test_float_float_exponential_constants():
    """Cody-Waite split of ln2/32 and 32/ln2 of the float-float exponential:
    c1, c2 short enough that n c1, n c2 are exact for every n the kernel
    forms (u <= 87), and c1 + c2 + c3 + c4 = ln2/32 to far below float-float
    precision."""
    c = _constexpr_floats("fsff.cu")
    c1, c2, c3, c4, inv = c["kC1"], c["kC2"], c["kC3"], c["kC4"], c["kInvL"]
    with mpmath.workdps(50):
        l32 = mpmath.log(2) / 32
        total = sum(mpmath.mpf(float(v)) for v in (c1, c2, c3, c4))
        assert abs(total / l32 - 1) < 1e-22  # 4.4e-24: the FP32 rounding of c4
        assert abs(mpmath.mpf(float(inv)) * l32 - 1) < 2 ** -24
    n_max = int(np.ceil(87.0 * float(inv)))
    assert n_max < 2 ** 13
    for v in (c1, c2):
        # n (< 2^13) times an 11-bit significand fits the 24-bit significand
        assert _significant_bits(v) <= 11
        for n in (1, 3, 4095, n_max):
            assert float(np.float32(n) * v) == n * float(v)
    # e^-r series cut after r^5: the remainder at |r| = ln2/64 (plus the
    # rounding of n) is 2.2e-15 relative, below the float-float precision
    # 2^-48 = 3.6e-15
    r = float(mpmath.log(2) / 64) * 1.001
    assert r ** 6 / 720 < 2 ** -48
