"""Pins of the oracle's binary16 / bfloat16 rounding (Table 1 storage formats).

The oracle rounds from the IEEE 754 definition (spacing of the binade,
nearbyint, gradual underflow, overflow to infinity).  It is checked against
independent sources: numpy's float16 conversion, torch's bfloat16 conversion,
the classic bit-level round-to-nearest-even formula for bfloat16, and
hand-worked values; fp32 -> fp16 / bf16 on every one of the 2^32 fp32 bit
patterns.
"""
import numpy as np
import pytest
import torch

import oracle as O
from problems import rng


def _samples():
    # every binary16 value, every midpoint between neighbours, and the
    # midpoints nudged by one fp64 ulp in both directions
    h = np.arange(0, 0x7C00, dtype=np.uint16).view(np.float16).astype(np.float64)
    mids = 0.5 * (h[:-1] + h[1:])
    vals = np.concatenate([h, mids, np.nextafter(mids, 0), np.nextafter(mids, np.inf),
                           [65504.0, 65519.999, 65520.0, 65536.0, 1e6, 2.0 ** -25, 2.0 ** -24,
                            3 * 2.0 ** -26, 2.0 ** -26]])
    u = rng.uniform01(5, 1, 200000)
    e = rng.integers(5, 2, 200000, -30, 20)
    rnd = (2 * u - 1) * np.exp2(e.astype(np.float64))
    vals = np.concatenate([vals, rnd])
    return np.concatenate([vals, -vals])


def test_f16_matches_numpy_float64_source(orc):
    x = _samples()
    want = x.astype(np.float16).astype(np.float64)  # numpy rounds double -> half directly
    got = O.round_to(O.F16, x)
    assert np.array_equal(np.signbit(got), np.signbit(want))
    assert np.array_equal(got, want)


def test_f16_matches_numpy_float32_source(orc):
    x = _samples().astype(np.float32)
    want = x.astype(np.float16).astype(np.float64)
    got = O.round_to(O.F16, x.astype(np.float64))
    assert np.array_equal(got, want)


def test_f16_hand_worked_values(orc):
    # ties go to the even neighbour; spacing is 2^-10 in [1, 2)
    cases = {
        1.0 + 2.0 ** -11: 1.0,                       # tie, 1.0 is even
        1.0 + 3 * 2.0 ** -11: 1.0 + 2 * 2.0 ** -10,  # tie, rounds up to even
        1.0 + 2.0 ** -11 + 2.0 ** -30: 1.0 + 2.0 ** -10,
        65519.0: 65504.0,
        65520.0: np.inf,                              # half-way to 2^16 overflows
        2.0 ** -24: 2.0 ** -24,                       # smallest subnormal
        2.0 ** -25: 0.0,                              # tie with zero goes to zero
        1.5 * 2.0 ** -25: 2.0 ** -24,
        -2.0 ** -26: -0.0,
    }
    x = np.array(list(cases.keys()))
    got = O.round_to(O.F16, x)
    want = np.array(list(cases.values()))
    assert np.array_equal(got, want)
    assert np.signbit(got[-1])


def _bf16_bits_rne(x32: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even of float32 bit patterns to the upper 16 bits."""
    b = x32.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16).astype(np.uint32) << 16
    return r.view(np.float32).astype(np.float64)


def test_bf16_matches_bit_formula_and_torch(orc):
    u = rng.uniform01(6, 1, 300000)
    e = rng.integers(6, 2, 300000, -140, 127)
    x = ((2 * u - 1) * np.exp2(e.astype(np.float64))).astype(np.float32)
    x = x[np.isfinite(x)]
    got = O.round_to(O.BF16, x.astype(np.float64))
    want_bits = _bf16_bits_rne(x)
    want_torch = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(got, want_bits)
    assert np.array_equal(got, want_torch)


def test_bf16_hand_worked_values(orc):
    cases = {
        1.0 + 2.0 ** -8: 1.0,                    # tie -> even
        1.0 + 3 * 2.0 ** -8: 1.0 + 2.0 ** -6,    # tie -> even (up)
        3.3895313892515355e38: 3.3895313892515355e38,
        3.3961775292304958e38: np.inf,           # half-way above the largest finite
    }
    x = np.array(list(cases.keys()))
    assert np.array_equal(O.round_to(O.BF16, x), np.array(list(cases.values())))


def test_f32_matches_numpy(orc):
    x = _samples() * 1.234567
    assert np.array_equal(O.round_to(O.F32, x), x.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("prec", [O.F16, O.BF16, O.F32])
def test_nonfinite_pass_through(orc, prec):
    x = np.array([np.inf, -np.inf, np.nan, 0.0, -0.0])
    y = O.round_to(prec, x)
    assert y[0] == np.inf and y[1] == -np.inf and np.isnan(y[2])
    assert y[3] == 0 and not np.signbit(y[3]) and np.signbit(y[4])


def test_every_float32_binade_and_sign_at_stride_256(orc):
    """fp32 -> fp16 and fp32 -> bf16 over the fp32 bit patterns at a stride of
    256 (every sign and exponent, every 256th significand, a seeded low byte):
    the oracle matches numpy's float16 cast and the bit-level bfloat16
    round-to-nearest-even formula on all 16.7 M finite inputs."""
    low = rng.integers(7, 1, 1, 0, 255)[0]
    bits = (np.arange(1 << 24, dtype=np.uint64) << np.uint64(8)) | np.uint64(low)
    x32 = bits.astype(np.uint32).view(np.float32)
    x32 = x32[np.isfinite(x32)]
    x64 = x32.astype(np.float64)
    got16 = O.round_to(O.F16, x64)
    with np.errstate(over="ignore"):
        want16 = x32.astype(np.float16).astype(np.float64)
    same = (got16 == want16) | (np.isnan(got16) & np.isnan(want16))
    assert np.all(same) and np.array_equal(np.signbit(got16), np.signbit(want16))
    gotbf = O.round_to(O.BF16, x64)
    assert np.array_equal(gotbf, _bf16_bits_rne(x32))


def _all_patterns_piece(start, count):
    """mismatches of the oracle's fp16 and bf16 rounding against numpy's fp16
    cast and the bit-level bf16 formula on fp32 patterns start .. start + count - 1"""
    u = (np.arange(start, start + count, dtype=np.uint64) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    x32 = u.view(np.float32)
    fin = np.isfinite(x32)
    x64 = x32.astype(np.float64)
    got16 = O.round_to(O.F16, x64)
    with np.errstate(over="ignore", invalid="ignore"):
        want16 = x32.astype(np.float16).astype(np.float64)
    bad = int(np.count_nonzero((got16 != want16) & fin))
    bad += int(np.count_nonzero(np.signbit(got16[fin]) != np.signbit(want16[fin])))
    gotbf = O.round_to(O.BF16, x64)
    bf = ((u + np.uint32(0x7FFF) + ((u >> np.uint32(16)) & np.uint32(1))) >> np.uint32(16)) << np.uint32(16)
    wantbf = bf.view(np.float32).astype(np.float64)
    bad += int(np.count_nonzero((gotbf != wantbf) & fin))
    # inf and nan in, the same out
    bad += int(np.count_nonzero(np.isnan(x64) != np.isnan(got16)) + np.count_nonzero(np.isnan(x64) != np.isnan(gotbf)))
    return bad


def test_every_float32_pattern(orc):
    """The oracle's fp32 -> fp16 and fp32 -> bf16 rounding against numpy's
    float16 cast and the bit-level round-to-nearest-even bfloat16 formula on
    all 2^32 fp32 bit patterns (NaN in, NaN out), in pieces across threads
    (the oracle's C loop and numpy release the interpreter lock)."""
    from concurrent.futures import ThreadPoolExecutor

    piece = 1 << 24
    with ThreadPoolExecutor(max_workers=8) as ex:
        bad = sum(ex.map(lambda s: _all_patterns_piece(s, piece), range(0, 1 << 32, piece)))
    assert bad == 0, bad
