"""The FP32 pair kernel forms the Box-Muller uniforms u = (2 (x >> 9) + 1) 2^-24
(the reading of the pair noise: odd multiples of 2^-24, never 0 or 1) from the
bits of a Philox output word without an integer-to-float conversion: the
binary32 number 1 + (x >> 9) 2^-23 is built by its bits, and 1 - 2^-24 is
subtracted from it.  That subtraction is exact (Sterbenz: the operands are
within a factor 2 of each other, and the result has at most 24 significant
bits), so the uniform is the defined value for every word.  This checks the
identity exhaustively over all 2^23 mantissas in IEEE binary32 arithmetic."""
import numpy as np


def test_uniform_from_one_subtraction_is_exact_for_every_mantissa():
    m = np.arange(1 << 23, dtype=np.uint32)
    one_plus = (np.uint32(0x3F800000) | m).view(np.float32)
    u = one_plus - np.float32(1.0 - 2.0 ** -24)
    want = (2.0 * m.astype(np.float64) + 1.0) * 2.0 ** -24
    assert u.dtype == np.float32
    assert np.array_equal(u.astype(np.float64), want)
    assert u.min() > 0.0 and u.max() < 1.0


def test_uniform_matches_the_word_it_comes_from():
    # x >> 9 keeps the top 23 bits of the word; the bottom 9 bits do not matter
    rng = np.random.default_rng(12)
    x = rng.integers(0, 1 << 32, 4096, dtype=np.uint64).astype(np.uint32)
    u = ((np.uint32(0x3F800000) | (x >> np.uint32(9))).view(np.float32)
         - np.float32(1.0 - 2.0 ** -24))
    want = (((x >> np.uint32(8)) | np.uint32(1)).astype(np.float64)) * 2.0 ** -24
    assert np.array_equal(u.astype(np.float64), want)
