"""The integer-pipe predicates of csrc/mhd_math.cuh, restated on numpy bit
patterns and checked against the plain floating-point definitions.

The kernels decide minmod, |x| < y and x < -y from the bit patterns of the
doubles (so that no FP64 instruction is spent on an absolute value or a
negation); these tests pin the identities those forms rest on, over random
doubles of every magnitude and sign, signed zeros, subnormals and infinities.
The GPU suite checks separately that the kernels' results did not change."""
import numpy as np


def bits(x):
    return np.asarray(x, dtype=np.float64).view(np.int64)


def sample(n=200_000, seed=3):
    rng = np.random.default_rng(seed)
    mant = rng.uniform(1.0, 2.0, n)
    expo = rng.integers(-1074, 1024, n)
    x = np.ldexp(mant, expo)                      # every binade, subnormals included
    x[rng.random(n) < 0.5] *= -1.0
    special = np.array([0.0, -0.0, np.inf, -np.inf, 5e-324, -5e-324, 1.0, -1.0, 2.0, -2.0])
    return np.concatenate([x, special, rng.choice(x, 50), rng.choice(special, 50)])


def minmod_reference(a, b):
    """0 when the signs differ or either is 0, else the argument of smaller magnitude (a on ties)."""
    out = np.where(np.abs(b) < np.abs(a), b, a)
    same_sign = (np.sign(a) == np.sign(b)) & (a != 0) & (b != 0)
    return np.where(same_sign, out, 0.0)


def minmod_bits(a, b):
    ia, ib = bits(a), bits(b)
    same = (ia ^ ib) >= 0
    return np.where(same, np.where(ib < ia, b, a), 0.0)


def test_minmod_from_signed_bit_patterns():
    x = sample()
    rng = np.random.default_rng(4)
    y = rng.permutation(x)
    got, want = minmod_bits(x, y), minmod_reference(x, y)
    # equal as values; where both are zero the kernel may return a signed zero of either input
    assert np.array_equal(got, want)
    nz = want != 0
    assert np.array_equal(bits(got[nz]), bits(want[nz]))


def test_same_sign_doubles_order_like_their_bits():
    x = sample()
    y = np.random.default_rng(5).permutation(x)
    same = (bits(x) ^ bits(y)) >= 0
    assert np.array_equal((np.abs(y) < np.abs(x))[same], (bits(y) < bits(x))[same])


def lt_abs_bits(x, y):
    ux = bits(x).view(np.uint64) << np.uint64(1)
    uy = bits(y).view(np.uint64) << np.uint64(1)
    return (bits(y) >= 0) & (ux < uy)


def test_lt_abs_is_the_masked_compare():
    """lt_abs(x, y) = lt_pos(|x|, y): bits(|x|) < bits(y) as signed integers, false for y < 0."""
    x = sample()
    y = np.random.default_rng(6).permutation(x)
    masked = (bits(x) & np.int64(0x7FFFFFFFFFFFFFFF)) < bits(y)
    assert np.array_equal(lt_abs_bits(x, y), masked)
    pos = (y >= 0) & ~np.isnan(y)
    assert np.array_equal(lt_abs_bits(x, y)[pos], (np.abs(x) < y)[pos])


def order_key(x):
    b = bits(x)
    return b ^ ((b >> 63) & np.int64(0x7FFFFFFFFFFFFFFF))


def test_order_key_of_minus_y_is_not_bits_y():
    """For y >= 0 (a square), key(-y) = ~bits(y), so x < -y needs no negation."""
    x = sample()
    y = np.abs(np.random.default_rng(7).permutation(x))
    assert np.array_equal(order_key(-y), ~bits(y))
    assert np.array_equal(order_key(x) < ~bits(y), x < -y)


def test_neg_if_flips_only_the_sign():
    x = sample()
    flipped = (bits(x) ^ np.int64(-0x8000000000000000)).view(np.float64)
    assert np.array_equal(bits(flipped), bits(-x))
