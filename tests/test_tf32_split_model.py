"""The TF32 split of the tensor-core GEMM operands, x = x_hi + x_lo.

The kernels form x_hi with integer operations on the bit pattern: half a TF32 unit (bit
12) added to the magnitude bits, then the 13 low bits cleared.  These tests check that
rule, restated here on numpy's uint32, against rounding to nearest with ties away from
zero onto the TF32 grid written from its definition (10 fraction bits: spacing
2^(e - 10) in the binade [2^e, 2^(e+1)), the binade of the smallest normal below it), and
that x_lo = x - x_hi is exact.  (On the GPU the same rule was compared with the
conversion instruction on all 2^32 inputs.)"""
import numpy as np


def split_bits(x):
    u = x.view(np.uint32)
    hi = ((u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).view(np.float32)
    return hi, (x - hi).astype(np.float32)


def round_tf32_definition(x):
    """Nearest TF32 value, ties away from zero, from the grid spacing (float64 arithmetic)."""
    x64 = x.astype(np.float64)
    ax = np.abs(x64)
    out = np.zeros_like(x64)
    nz = ax > 0
    _, e = np.frexp(ax[nz])                       # ax = m 2^e, m in [0.5, 1)
    lead = np.maximum(e - 1, -126)                # leading binade, subnormals share -126
    spacing = np.ldexp(1.0, lead - 10)
    q = ax[nz] / spacing                          # exact: at most 24 significant bits
    r = np.floor(q + 0.5)
    out[nz] = np.sign(x64[nz]) * r * spacing
    with np.errstate(over="ignore"):
        res = out.astype(np.float32)
    res[~nz] = x[~nz]                             # signed zeros unchanged
    return res


def _edge_values():
    bits = [0x00000000, 0x80000000, 0x00000001, 0x00001000, 0x00001FFF, 0x00002000,
            0x007FFFFF, 0x00800000, 0x00801000, 0x00800FFF, 0x3F800000, 0x3F801000,
            0x3F800FFF, 0x3F801001, 0x3FFFF000, 0x3FFFFFFF, 0x7F7FEFFF, 0x7F7FF000,
            0xBF801000, 0xBFFFF000, 0xFF7FEFFF]
    return np.array(bits, np.uint32).view(np.float32)


def test_integer_rounding_is_round_to_nearest_ties_away():
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 2 ** 32, size=1 << 20, dtype=np.uint64).astype(np.uint32)
    x = np.concatenate([bits.view(np.float32), _edge_values()])
    x = x[np.isfinite(x)]
    hi, _ = split_bits(x)
    ref = round_tf32_definition(x)
    np.testing.assert_array_equal(hi.view(np.uint32), ref.view(np.uint32))


def test_ties_round_away_from_zero():
    # bit 12 set, bits 0-11 clear: exactly half a TF32 unit above a grid point
    x = np.array([0x3F801000, 0xBF801000, 0x00801000], np.uint32).view(np.float32)
    hi, _ = split_bits(x)
    assert list(hi.view(np.uint32)) == [0x3F802000, 0xBF802000, 0x00802000]


def test_low_part_is_exact_and_small():
    rng = np.random.default_rng(1)
    x = (rng.normal(size=1 << 18) * np.exp(rng.uniform(-60, 60, 1 << 18))).astype(np.float32)
    hi, lo = split_bits(x)
    assert np.all((hi.view(np.uint32) & np.uint32(0x1FFF)) == 0)
    np.testing.assert_array_equal(hi + lo, x)
    nz = x != 0
    assert np.all(np.abs(lo[nz]) <= np.abs(x[nz]) * 2.0 ** -11 * (1 + 2.0 ** -10))


def test_largest_values_round_to_infinity_like_the_grid():
    x = np.array([0x7F7FF000, 0x7F7FFFFF], np.uint32).view(np.float32)
    hi, _ = split_bits(x)
    assert np.all(np.isinf(hi))
    assert np.all(np.isinf(round_tf32_definition(x)))
