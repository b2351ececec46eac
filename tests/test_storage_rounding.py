"""Pins of the storage roundings that the low-precision form uploads.

`inputs.to_f32` and `inputs.bf16_bits` produce the FP32 and BF16 value
arrays that the binding uploads and that the precision tests dequantise to
build their "stored" reference, so both sides share them.  A truncating or
mis-tied rounding would move both sides together and still pass a loose
check against the original FP64 values, so each one is pinned here against
an independent round-to-nearest-even: numpy's float64 -> float32 cast and
torch's float32 -> bfloat16 cast, plus hand-worked tie cases.  No GPU.
"""
import numpy as np
import pytest

from paper_2209_07552_gb300 import inputs as I


def _f32_of_bits(bits):
    return np.asarray(bits, np.uint32).view(np.float32).astype(np.float64)


def test_to_f32_is_numpy_nearest_even():
    g = np.random.default_rng(7)
    v = g.standard_normal(200_000) * np.exp2(g.integers(-140, 120, 200_000))
    assert np.array_equal(I.to_f32(v).view(np.uint32), v.astype(np.float32).view(np.uint32))
    # exact ties between two binary32 neighbours: 1 + 2^-24 lies halfway
    # between 1 and 1 + 2^-23; nearest-even keeps 1 (even mantissa), while
    # 1 + 3*2^-24 goes up to 1 + 2^-22 (even)
    assert I.to_f32(np.array([1.0 + 2.0**-24]))[0] == np.float32(1.0)
    assert I.to_f32(np.array([1.0 + 3 * 2.0**-24]))[0] == np.float32(1.0 + 2.0**-22)


@pytest.mark.parametrize("bits, want", [
    (0x3F808000, 0x3F80),  # halfway, mantissa of the lower neighbour even: stays
    (0x3F818000, 0x3F82),  # halfway, lower neighbour odd: rounds up to even
    (0x3F808001, 0x3F81),  # just above halfway: up
    (0x3F807FFF, 0x3F80),  # just below halfway: down
    (0xBF818000, 0xBF82),  # the same tie, negative: magnitude rounds to even
    (0x3F800000, 0x3F80),  # exact
    (0x00000000, 0x0000),  # +0
    (0x80000000, 0x8000),  # -0
    (0x00018000, 0x0002),  # subnormal tie, lower neighbour odd: up
    (0x00008000, 0x0000),  # subnormal tie, lower neighbour even (zero): stays
    (0x7F7FFFFF, 0x7F80),  # largest binary32 rounds to bfloat16 infinity
    (0x7F7F7FFF, 0x7F7F),  # below the halfway point to infinity: stays finite
])
def test_bf16_bits_hand_worked_ties(bits, want):
    assert int(I.bf16_bits(_f32_of_bits([bits]))[0]) == want


def test_bf16_bits_matches_torch_cast():
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(11)
    # random binary32 patterns over all finite exponents, and values of the
    # generators' own ranges (U(-1, 1), N(0, 1), products of both)
    pat = g.integers(0, 1 << 32, 400_000, dtype=np.uint64).astype(np.uint32)
    pat = pat[(pat & 0x7F800000) != 0x7F800000]  # no inf / NaN inputs
    vals = np.concatenate([
        pat.view(np.float32).astype(np.float64),
        g.uniform(-1, 1, 100_000),
        g.standard_normal(100_000),
        g.uniform(-1, 1, 100_000) * g.standard_normal(100_000),
    ])
    f32 = vals.astype(np.float32)
    want = torch.from_numpy(f32).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    got = I.bf16_bits(vals)
    assert np.array_equal(got, want)


def test_bf16_round_trip_is_the_nearest_bfloat16():
    """bf16_to_f32(bf16_bits(v)) is a nearest representable bfloat16 of the
    binary32 value: no other bfloat16 is closer (brute force over the two
    neighbours)."""
    g = np.random.default_rng(13)
    v = g.standard_normal(50_000)
    f = I.to_f32(v).astype(np.float64)
    b = I.bf16_bits(v)
    q = I.bf16_to_f32(b).astype(np.float64)
    up = I.bf16_to_f32((b.astype(np.int32) + 1).astype(np.uint16)).astype(np.float64)
    dn = I.bf16_to_f32((b.astype(np.int32) - 1).astype(np.uint16)).astype(np.float64)
    assert np.all(np.abs(f - q) <= np.abs(f - up))
    assert np.all(np.abs(f - q) <= np.abs(f - dn))
