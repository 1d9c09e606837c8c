"""Host checks of the exact digit arithmetic behind the tensor-core contractions (the scheme the
kernels of theta_tc.cu implement; emulated here in numpy, no GPU).

float64 path: a value |x| < 2^(rho - 1) becomes q = round(x 2^(55 - rho)), |q| < 2^54, written as
seven balanced base-256 digits in [-128, 127] (0x80 added to every byte of q, subtracted again per
digit); products of digit levels s = i + j <= 6 are kept.  float32 path: q = round(256 round_1)
with round_1 the nearest integer of x 2^21 (the magic-constant FMA 1.5 2^23), four digits, levels
s <= 3.  The checks: the digits are balanced and reconstruct q exactly; the kept levels reproduce
the product to the stated fraction of the operands' bounds; a level's sum over the stated number
of degrees (or rings) stays an exact float32 integer.
"""
import numpy as np

MAGIC = np.float32(12582912.0)        # 1.5 * 2^23


def _fma32(a, b, c):
    """float32 fused multiply-add: the exact a*b + c (held in float64 here, where every product
    of two float32 values and the small sums below are exact) rounded once to float32."""
    return np.float32(np.float64(a) * np.float64(b) + np.float64(c))


def split32(x, scale):
    """The float32 kernels' split: (q, digits most significant first), q ~ x * scale * 256."""
    y1 = _fma32(x, scale, MAGIC)
    hi = np.float32(y1 - MAGIC)
    y2 = _fma32(_fma32(x, scale, -hi), np.float32(256.0), MAGIC)
    q = (int(y1.view(np.uint32)) - 0x4B400000) * 256 + (int(y2.view(np.uint32)) - 0x4B400000)
    qo = (q + 0x80808080) & 0xFFFFFFFF
    return q, [((qo >> (8 * p)) & 0xFF) - 128 for p in (3, 2, 1, 0)]


def split64(x, rho):
    """The float64 kernels' split: q = round(x 2^(55 - rho)) and its seven balanced digits."""
    q = int(np.rint(np.ldexp(np.float64(x), 55 - rho)))
    qo = (q + 0x0080808080808080) & 0xFFFFFFFFFFFFFFFF
    return q, [((qo >> (8 * p)) & 0xFF) - 128 for p in range(6, -1, -1)]


def _kept(dx, dy, nd, smax):
    """sum over i + j <= smax of dx_i dy_j 256^(2 (nd - 1) - i - j)."""
    return sum(dx[i] * dy[j] * 256 ** (2 * (nd - 1) - i - j)
               for i in range(nd) for j in range(nd) if i + j <= smax)


def test_float32_split_digits_and_error():
    rng = np.random.default_rng(0)
    worst = 0.0
    for _ in range(4000):
        d = np.float32(rng.uniform(-1, 1))                # |d| <= 1: scale 2^21
        h = np.float32(rng.standard_normal() * 10.0 ** rng.integers(-20, 20))
        eps = int(np.floor(np.log2(abs(float(h))))) + 1   # |h| < 2^eps
        qd, dd = split32(d, np.float32(2.0 ** 21))
        qh, hh = split32(h, np.float32(2.0 ** (21 - eps)))
        for q, dig in ((qd, dd), (qh, hh)):
            assert all(-128 <= v <= 127 for v in dig)
            assert q == sum(v * 256 ** (3 - i) for i, v in enumerate(dig))
            assert abs(q) <= 2 ** 29 + 128
        assert abs(qd - float(d) * 2.0 ** 29) <= 0.5 + 1e-9
        val = _kept(dd, hh, 4, 3) * 2.0 ** (eps - 58)
        worst = max(worst, abs(val - float(d) * float(h)) / 2.0 ** eps)
    assert worst < 2.0 ** -26                                # measured 8.6e-9 = 2^-26.8


def test_three_float32_digits_would_not_reach_float32_accuracy():
    """With 24 bits (three digits, levels <= 2) the dropped level weighs ~2^-20: the reason the
    float32 kernel carries four digits."""
    rng = np.random.default_rng(1)
    worst = 0.0
    for _ in range(4000):
        d = float(rng.uniform(-1, 1))
        h = float(rng.standard_normal())
        eps = int(np.floor(np.log2(abs(h)))) + 1
        def dig3(q):
            qo = (q + 0x808080) & 0xFFFFFF
            return [((qo >> (8 * p)) & 0xFF) - 128 for p in (2, 1, 0)]
        a = dig3(int(np.rint(d * 2 ** 21)))
        b = dig3(int(np.rint(h * 2 ** (21 - eps))))
        val = _kept(a, b, 3, 2) * 2.0 ** (eps - 42)
        worst = max(worst, abs(val - d * h) / 2.0 ** eps)
    assert worst > 2.0 ** -21


def test_float64_split_digits_and_error():
    rng = np.random.default_rng(2)
    worst = 0.0
    for _ in range(3000):
        x = rng.uniform(-1, 1) * 2.0 ** rng.integers(-30, 0)
        y = rng.uniform(-1, 1)
        rx, ry = 2, 2                                       # |x|, |y| < 2^(rho - 1) = 2
        qx, dx = split64(x, rx)
        qy, dy = split64(y, ry)
        for q, dig in ((qx, dx), (qy, dy)):
            assert all(-128 <= v <= 127 for v in dig)
            assert q == sum(v * 256 ** (6 - i) for i, v in enumerate(dig))
            assert abs(q) < 2 ** 54
        val = _kept(dx, dy, 7, 6) * 2.0 ** (rx + ry - 110)
        worst = max(worst, abs(val - x * y) / 4.0)
    assert worst < 2.0 ** -52


def test_level_sums_stay_exact_in_float32():
    """A level receives at most (number of digits) products of magnitude <= 2^14 per term: the
    float64 inverse (7 digits) reads back every 128 degrees, the float32 inverse (4 digits) every
    128 degrees, the float64 forward sums 256 rings per tile for each digit pair separately."""
    assert 7 * 2 ** 14 * 128 < 2 ** 24
    assert 4 * 2 ** 14 * 128 <= 2 ** 23
    assert 256 * 2 ** 14 <= 2 ** 22
    # and the worst case of balanced digits is 128 * 128 = 2^14
    assert max(abs(a * b) for a in (-128, 127) for b in (-128, 127)) == 2 ** 14
