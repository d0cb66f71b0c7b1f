"""Exactness of the fixed-point fold of the FP64-class digit products.

The FP64-class updates write each operand entry as 8 digits of 7 bits
(|digit 0| <= 128, |digit p| <= 64 for p >= 1), accumulate the 36 digit
products with p + q < 8 in 8 FP32 group sums over at most 256 K terms, and
fold the groups per chunk in integer arithmetic:
  T = sum_{g>=2} G_g 2^(7(7-g))   (64-bit Horner),
  Q = 2^7 G_0 + G_1               (32-bit),
  hi += 2^10 Q + floor(T / 2^32),  lo += T mod 2^32 (32-bit word, carry into hi),
so that the chunk's value is Q 2^-21 + T 2^-63 = hi 2^-31 + lo 2^-63.
These checks restate those bounds and identities with Python integers: every
group sum fits FP32 exactly, T fits a signed 64-bit word, Q a signed 32-bit
word, and the (hi, lo) accumulator reproduces sum_chunks sum_g G_g 2^-7(g+2)
exactly.  No GPU is needed.
"""
import random
from fractions import Fraction

NS, BITS, KCHUNK = 8, 7, 256


def group_bound(g: int) -> int:
    """Largest |G_g| over KCHUNK terms: products of digit pairs with p + q = g."""
    per_term = 0
    for p in range(g + 1):
        q = g - p
        if p >= NS or q >= NS:
            continue
        da = 128 if p == 0 else 64
        db = 128 if q == 0 else 64
        per_term += da * db
    return KCHUNK * per_term


def fold(groups):
    t = groups[2]
    for g in range(3, NS):
        t = t * 128 + groups[g]
    q = groups[0] * 128 + groups[1]
    return q, t


def test_group_sums_are_exact_in_fp32():
    for g in range(NS):
        assert group_bound(g) < 2 ** 24, g
    # the stated bounds: |G_0| <= 2^22, |G_g| < 2^23.4 for g >= 1
    assert group_bound(0) == 2 ** 22
    assert max(group_bound(g) for g in range(1, NS)) < 2 ** 23.4


def test_fold_words_do_not_overflow():
    worst = [group_bound(g) for g in range(NS)]
    q, t = fold(worst)
    assert abs(t) < 2 ** 59 < 2 ** 63
    assert abs(q) < 2 ** 30 < 2 ** 31
    qn, tn = fold([-w for w in worst])
    assert abs(tn) < 2 ** 59 and abs(qn) < 2 ** 30


def test_fixed_point_accumulator_is_exact():
    rng = random.Random(7)
    for trial in range(200):
        nchunks = rng.randint(1, 80)
        hi, lo = 0, 0  # lo: an unsigned 32-bit word
        exact = Fraction(0)
        for _ in range(nchunks):
            groups = [rng.randint(-group_bound(g), group_bound(g)) for g in range(NS)]
            exact += sum(Fraction(groups[g], 2 ** (BITS * (g + 2))) for g in range(NS))
            q, t = fold(groups)
            # the device code: l = lo + (unsigned) t (mod 2^32), carry when it wraps
            l = (lo + (t & 0xFFFFFFFF)) & 0xFFFFFFFF
            carry = 1 if l < lo else 0
            hi += q * 1024 + (t >> 32) + carry  # arithmetic shift: floor
            lo = l
            assert -(2 ** 63) < hi < 2 ** 63
        assert Fraction(hi, 2 ** 31) + Fraction(lo, 2 ** 63) == exact, trial
