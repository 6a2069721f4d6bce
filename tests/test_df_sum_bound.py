"""The compensated double-float hopping sums of both passes, replayed with numpy float32
arithmetic on the host, against their derived error bounds (no GPU).

The sum keeps H, the FP32 running sum of the high words, exact by TwoSum, sums H's rounding
errors exactly as well (a second TwoSum into L, whose own errors go to C), adds the low words
plainly into four accumulators used in turn, and closes with TwoSums and one rounding.  Its
error over F terms of total magnitude A is at most (N - 1 + 1.01) 2^-48 A, N the most terms one
low-word accumulator takes (ceil(F/4) for one sign group).  Replayed here on inputs built to
maximise the rounding (one-signed maximal low words, large partial sums, random orders), with
the exact sum taken in Python fractions; the plain form (errors and low words in one FP32
word) is replayed beside it and shown to exceed its own first-order budget by far."""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32
U2 = 2.0 ** -48


def _two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    e = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, e


def _compensated(hi, lo):
    H = L = C = f32(0.0)
    V = [f32(0.0)] * 4
    for k, (h, l) in enumerate(zip(hi, lo)):
        H, e = _two_sum(H, h)
        L, f = _two_sum(L, e)
        C = f32(C + f)
        V[k % 4] = f32(V[k % 4] + l)
    for j in range(4):
        L, f = _two_sum(L, V[j])
        C = f32(C + f)
    s, e = _two_sum(H, L)
    h, l = _two_sum(s, f32(e + C))
    return Fraction(float(h)) + Fraction(float(l))


def _paired(hi, lo):
    """Pass 2's form: the same H, L, C chain, the low parts of two terms added together (one
    rounding) and the pair sums going to two accumulators: in batches of four terms the first
    pair to accumulator 0 and the second to 1, a last pair to 0, a last single term to 1."""
    H = L = C = f32(0.0)
    V = [f32(0.0)] * 2

    def hi_step(h):
        nonlocal H, L, C
        H, e = _two_sum(H, h)
        L, f = _two_sum(L, e)
        C = f32(C + f)

    F, k = len(hi), 0
    while k + 4 <= F:
        for q, j in ((k, 0), (k + 2, 1)):
            hi_step(hi[q])
            hi_step(hi[q + 1])
            V[j] = f32(V[j] + f32(lo[q] + lo[q + 1]))
        k += 4
    if k + 2 <= F:
        hi_step(hi[k])
        hi_step(hi[k + 1])
        V[0] = f32(V[0] + f32(lo[k] + lo[k + 1]))
        k += 2
    if k < F:
        hi_step(hi[k])
        V[1] = f32(V[1] + lo[k])
    for j in range(2):
        L, f = _two_sum(L, V[j])
        C = f32(C + f)
    s, e = _two_sum(H, L)
    h, l = _two_sum(s, f32(e + C))
    return Fraction(float(h)) + Fraction(float(l))


def _plain(hi, lo):
    H = L = f32(0.0)
    for h, l in zip(hi, lo):
        H, e = _two_sum(H, h)
        L = f32(f32(L + l) + e)
    s, e = _two_sum(H, L)
    return Fraction(float(s)) + Fraction(float(e))


def _split(x):
    """Normalised double-float pair of a float64 (|lo| <= 2^-24 |hi|)."""
    hi = x.astype(f32)
    lo = (x - hi.astype(np.float64)).astype(f32)
    return hi, lo


def _adversarial(rng, F):
    """Positive terms: one large first term and F - 1 of magnitude 2^U[-6, 0] with random
    high-word bits and low words of nearly half a unit in the last place, all one-signed."""
    e = rng.integers(-6, 1, F).astype(np.float64)
    m = 1.0 + rng.integers(0, 1 << 23, F) / float(1 << 23)
    hi = np.ldexp(m, e.astype(int))
    hi[0] = 2.0 ** 5
    x = hi + np.ldexp(0.4999, e.astype(int) - 23)
    return x


@pytest.mark.parametrize("F", [8, 17, 32])
def test_compensated_sum_within_derived_bound(F):
    rng = np.random.default_rng(F)
    N = -(-F // 4)
    worst = 0.0
    for trial in range(300):
        x = _adversarial(rng, F) if trial % 2 == 0 else rng.normal(size=F) * 10.0 ** rng.uniform(-3, 0, F)
        hi, lo = _split(x)
        if trial % 3 == 0:
            p = rng.permutation(F)
            hi, lo = hi[p], lo[p]
        exact = sum(Fraction(float(h)) + Fraction(float(l)) for h, l in zip(hi, lo))
        A = float(sum(abs(Fraction(float(h)) + Fraction(float(l))) for h, l in zip(hi, lo)))
        err = abs(float(_compensated(hi, lo) - exact))
        worst = max(worst, err / (U2 * A))
        assert err <= (N - 1 + 1.01) * U2 * A, (trial, err / (U2 * A))
    print(f"F = {F}: worst error {worst:.3f} u^2 A (bound {N - 1 + 1.01:.2f})")


@pytest.mark.parametrize("F", [7, 8, 17, 32])
def test_paired_sum_within_derived_bound(F):
    """Pass 2's paired form: at most N = ceil(F/4) pair sums per low-part accumulator, so its
    error is at most (N - 1 + 1 + 1.01) u^2 A: the accumulators' roundings, one rounding per
    pair sum (u |vl_a + vl_b|, at most u^2 A over all pairs) and the closing."""
    rng = np.random.default_rng(100 + F)
    N = -(-F // 4)
    worst = 0.0
    for trial in range(300):
        x = _adversarial(rng, F) if trial % 2 == 0 else rng.normal(size=F) * 10.0 ** rng.uniform(-3, 0, F)
        hi, lo = _split(x)
        if trial % 3 == 0:
            p = rng.permutation(F)
            hi, lo = hi[p], lo[p]
        exact = sum(Fraction(float(h)) + Fraction(float(l)) for h, l in zip(hi, lo))
        A = float(sum(abs(Fraction(float(h)) + Fraction(float(l))) for h, l in zip(hi, lo)))
        err = abs(float(_paired(hi, lo) - exact))
        worst = max(worst, err / (U2 * A))
        assert err <= (N + 1.01) * U2 * A, (trial, err / (U2 * A))
    print(f"F = {F}: worst error {worst:.3f} u^2 A (bound {N + 1.01:.2f})")


def test_plain_sum_exceeds_linear_budget():
    """The uncompensated form's error grows faster than linearly in F: on the adversarial
    inputs it exceeds the (N - 1 + 1.01) u^2 A budget the compensated form keeps."""
    rng = np.random.default_rng(7)
    F, N = 32, 8
    worst = 0.0
    for _ in range(300):
        hi, lo = _split(_adversarial(rng, F))
        exact = sum(Fraction(float(h)) + Fraction(float(l)) for h, l in zip(hi, lo))
        A = float(sum(abs(Fraction(float(h)) + Fraction(float(l))) for h, l in zip(hi, lo)))
        worst = max(worst, abs(float(_plain(hi, lo) - exact)) / (U2 * A))
    assert worst > N - 1 + 1.01
