"""The library's fp32 -> fp16 / bf16 store conversion (f3r_round16: the
conversion every kernel applies when it stores a 16-bit value) on the GPU,
over every fp32 bit pattern (2^32 inputs), against definitions that share no
code with it:
* fp16: numpy's IEEE binary16 cast (round to nearest, ties to even,
  subnormals kept, overflow to infinity);
* bf16: round to nearest even on the bit pattern, (u + 0x7fff + lsb) >> 16,
  in numpy integer arithmetic;
and against the oracle's own bit-level rounding on a sample of about a
million patterns spread over every sign and binade, plus the special values.
A NaN input must give a NaN (payloads are not compared); every other input
must give the same 16-bit pattern.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2505_20719_gb300 import f3r  # noqa: E402

CHUNK = 1 << 27   # patterns per device launch (512 MB of fp32 input)
PIECE = 1 << 23   # patterns per host thread task


def _patterns_dev(start, count):
    """fp32 values whose bit patterns are start .. start + count - 1 (on the device)."""
    a = torch.arange(start, start + count, dtype=torch.int64, device="cuda")
    a = torch.where(a >= 2 ** 31, a - 2 ** 32, a).to(torch.int32)
    return a.view(torch.float32)


def _ref_piece(prec, start, got, lo, hi):
    """Compare got[lo:hi] (uint16) with the reference for patterns start+lo .. start+hi-1;
    returns the number of mismatches."""
    u = (np.arange(start + lo, start + hi, dtype=np.uint64) & 0xFFFFFFFF).astype(np.uint32)
    x = u.view(np.float32)
    nan = np.isnan(x)
    if prec == f3r.F16:
        with np.errstate(over="ignore", invalid="ignore"):
            ref = x.astype(np.float16).view(np.uint16)
        g = got[lo:hi]
        gnan = ((g & 0x7C00) == 0x7C00) & ((g & 0x03FF) != 0)
    else:
        ref = ((u + np.uint32(0x7FFF) + ((u >> np.uint32(16)) & np.uint32(1))) >> np.uint32(16)).astype(np.uint16)
        g = got[lo:hi]
        gnan = ((g & 0x7F80) == 0x7F80) & ((g & 0x007F) != 0)
    bad = int(np.count_nonzero((g != ref) & ~nan))
    bad += int(np.count_nonzero(nan != gnan))
    return bad


@pytest.mark.parametrize("prec", [f3r.F16, f3r.BF16], ids=["fp16", "bf16"])
def test_store_conversion_every_fp32_pattern(prec):
    out = torch.empty(CHUNK, dtype=torch.int16, device="cuda")
    host = torch.empty(CHUNK, dtype=torch.int16).pin_memory()
    bad = 0
    with ThreadPoolExecutor(max_workers=8) as ex:
        for start in range(0, 1 << 32, CHUNK):
            x = _patterns_dev(start, CHUNK)
            f3r.round16(prec, x, out)
            host.copy_(out)
            torch.cuda.synchronize()
            got = host.numpy().view(np.uint16).copy()
            bad += sum(ex.map(lambda lo: _ref_piece(prec, start, got, lo, lo + PIECE), range(0, CHUNK, PIECE)))
            del x
    assert bad == 0, bad


@pytest.mark.parametrize("prec", [f3r.F16, f3r.BF16], ids=["fp16", "bf16"])
def test_store_conversion_matches_oracle_rounding(prec):
    """The GPU conversion equals the oracle's round-to-16-bit on about a
    million patterns (a prime stride through all 2^32, every sign and binade)
    and on zeros, infinities, the largest finite values, the smallest
    normals and subnormals, and the values halfway between 16-bit neighbours."""
    pats = np.arange(0, 1 << 32, 4093, dtype=np.uint64)
    specials = [0x00000000, 0x80000000, 0x7F800000, 0xFF800000, 0x7F7FFFFF, 0xFF7FFFFF, 0x00800000, 0x80800000,
                0x00000001, 0x80000001, 0x33800000, 0x33000000, 0x387FC000, 0x38800000, 0x477FE000, 0x477FF000,
                0x477FEFFF, 0x3F808000, 0x3F818000, 0x7F7F8000, 0x7F7F7FFF]
    pats = np.concatenate([pats, np.array(specials, dtype=np.uint64)]).astype(np.uint32)
    x = pats.view(np.float32)
    xd = torch.from_numpy(x.copy()).cuda()
    out = torch.empty(x.size, dtype=torch.int16, device="cuda")
    f3r.round16(prec, xd, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint16)
    nan = np.isnan(x)
    y = O.round_to(O.F16 if prec == f3r.F16 else O.BF16, x[~nan].astype(np.float64))
    if prec == f3r.F16:
        with np.errstate(over="ignore"):
            ref = y.astype(np.float16).view(np.uint16)   # y is an fp16 value: exact
    else:
        ref = (y.astype(np.float32).view(np.uint32) >> np.uint32(16)).astype(np.uint16)  # y is a bf16 value
    assert np.array_equal(got[~nan], ref)
    gn = got[nan]
    if prec == f3r.F16:
        assert np.all(((gn & 0x7C00) == 0x7C00) & ((gn & 0x03FF) != 0))
    else:
        assert np.all(((gn & 0x7F80) == 0x7F80) & ((gn & 0x007F) != 0))


def test_round16_rejects_bad_arguments():
    x = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.empty(4, dtype=torch.int16, device="cuda")
    with pytest.raises(f3r.F3RError):
        f3r.round16(f3r.F32, x, out)
