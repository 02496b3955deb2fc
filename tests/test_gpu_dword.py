"""The double-word primitives of csrc/dword.cuh on the GPU against exact
rational arithmetic.

tests/dword_probe.cu evaluates, for seeded pairs (a, b) of binary64 values,
x = dw(a), y = dw(b), x + y, x - y, x * y, 1/y, sqrt(|x|), the Dot2 sum
x y + y y - x x + y and dw_to_double(x).  Each result is compared with the
exact value of the same operation on the double-word inputs (Fractions of the
FP32 words), against the error bound of its algorithm, u = 2^-24:

- conversion: the six dropped bits of the 52-bit fraction, < 2^-46 |a|;
- back to binary64: one rounding of h + l, <= 2^-53 |h + l|;
- sum (the "sloppy" double-word sum of Joldes, Muller & Popescu): relative
  3u^2 (to first order) for operands of one sign; absolute 8u^2 (|x| + |y|)
  under cancellation, above the first-order sum of its roundings (7u^2);
- product (2Prod of the high words plus the two cross terms by FMA, x_l y_l
  dropped): 6u^2 to first order, 6.5u^2 tested;
- reciprocal (one Newton step on the FP32 approximation, itself within about
  2^-22): 2^-43 relative; square root (one Newton step from x rsqrt(x), whose
  correction also carries the rsqrt error): 2^-42 relative;
- Dot2 accumulation: 10u^2 times the sum of the magnitudes of its terms, plus
  2u^2 of the result.

Inputs: magnitudes 10^U(-6, 6), mixed signs, and pairs that cancel to 1e-12 in
a sum or a difference.  A mistake in any error-free transformation (a
dropped correction term, a wrong operand order in 2Sum) gives errors near u,
2^36 times these bounds.
"""
import os
import shutil
import subprocess
from fractions import Fraction

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

U2 = Fraction(1, 2 ** 48)
HERE = os.path.dirname(os.path.abspath(__file__))


def _inputs(n=4000, seed=11):
    rng = np.random.default_rng(seed)
    m = n // 4
    mag = lambda k: 10.0 ** rng.uniform(-6, 6, k)
    a0, b0 = mag(m), mag(m)
    a1, b1 = mag(m) * rng.choice([-1.0, 1.0], m), mag(m) * rng.choice([-1.0, 1.0], m)
    a2 = mag(m) * rng.choice([-1.0, 1.0], m)
    b2 = -a2 * (1.0 + rng.choice([-1.0, 1.0], m) * 10.0 ** rng.uniform(-12, -3, m))   # x + y cancels
    a3 = mag(m) * rng.choice([-1.0, 1.0], m)
    b3 = a3 * (1.0 + rng.choice([-1.0, 1.0], m) * 10.0 ** rng.uniform(-12, -3, m))    # x - y cancels
    return np.concatenate([a0, a1, a2, a3]), np.concatenate([b0, b1, b2, b3])


@pytest.fixture(scope="module")
def probe_out(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    tmp = tmp_path_factory.mktemp("dword")
    exe = str(tmp / "dword_probe")
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-o", exe,
                    os.path.join(HERE, "dword_probe.cu")], check=True)
    a, b = _inputs()
    n = a.size
    with open(tmp / "in.bin", "wb") as f:
        f.write(np.int32(n).tobytes())
        f.write(a.astype("<f8").tobytes())
        f.write(b.astype("<f8").tobytes())
    subprocess.run([exe, str(tmp / "in.bin"), str(tmp / "out.bin")], check=True)
    raw = open(tmp / "out.bin", "rb").read()
    words = np.frombuffer(raw[: n * 16 * 4], dtype="<f4").reshape(n, 8, 2)
    back = np.frombuffer(raw[n * 16 * 4:], dtype="<f8")
    return a, b, words, back


def _val(w):
    return Fraction(float(w[0])) + Fraction(float(w[1]))


def test_conversions(probe_out):
    a, b, words, back = probe_out
    for i in range(a.size):
        for k, v in ((0, a[i]), (1, b[i])):
            assert abs(_val(words[i, k]) - Fraction(v)) < Fraction(1, 2 ** 46) * abs(Fraction(v)), (i, k)
        x = _val(words[i, 0])
        assert abs(Fraction(float(back[i])) - x) <= Fraction(1, 2 ** 53) * abs(x), i


def test_sum_and_difference(probe_out):
    a, _, words, _ = probe_out
    for i in range(a.size):
        x, y = _val(words[i, 0]), _val(words[i, 1])
        for k, exact in ((2, x + y), (3, x - y)):
            err = abs(_val(words[i, k]) - exact)
            assert err <= 8 * U2 * (abs(x) + abs(y)), (i, k)
            same_sign = (x > 0) == (y > 0) if k == 2 else (x > 0) != (y > 0)
            if same_sign:
                assert err <= Fraction(31, 10) * U2 * abs(exact), (i, k)


def test_product_reciprocal_sqrt(probe_out):
    a, _, words, _ = probe_out
    for i in range(a.size):
        x, y = _val(words[i, 0]), _val(words[i, 1])
        assert abs(_val(words[i, 4]) - x * y) <= Fraction(13, 2) * U2 * abs(x * y), i
        assert abs(_val(words[i, 5]) * y - 1) <= Fraction(1, 2 ** 43), i
        s = _val(words[i, 6])
        assert abs(s * s - abs(x)) <= 2 * Fraction(1, 2 ** 42) * abs(x), i     # 2 x relative error of s


def test_dot2_accumulation(probe_out):
    a, _, words, _ = probe_out
    for i in range(a.size):
        x, y = _val(words[i, 0]), _val(words[i, 1])
        terms = (x * y, y * y, -x * x, y)
        exact = sum(terms)
        err = abs(_val(words[i, 7]) - exact)
        assert err <= 10 * U2 * sum(abs(t) for t in terms) + 2 * U2 * abs(exact), i
