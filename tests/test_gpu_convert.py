"""The integer-pipe binary64 <-> binary32 conversions of the FP32 V-cycle kernels
against the hardware conversions (torch's casts on the GPU) and IEEE 754
round-to-nearest-even on the host (numpy's casts), bit for bit.

Inputs: every kind of binary64 encoding (uniform random bit patterns, which
are mostly outside binary32's range), random values inside binary32's normal
range, exact ties with even and odd kept fractions, the overflow boundary,
results that are binary32 subnormals, zeros, infinities and NaNs; for the
widening, uniform random 32-bit patterns and the special values.
"""

import ctypes as C

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2406_19754_gb300 import _lib

    return _lib.load()


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _narrow(x64):
    xd = torch.as_tensor(x64, device="cuda")
    out = torch.empty(xd.shape, dtype=torch.float32, device="cuda")
    assert _lib().amg_debug_convert(C.c_void_p(xd.data_ptr()), C.c_void_p(out.data_ptr()),
                                    None, None, xd.numel(), _stream()) == 0
    hw = xd.to(torch.float32)
    torch.cuda.synchronize()
    return out.cpu().numpy(), hw.cpu().numpy()


def _widen(x32):
    xd = torch.as_tensor(x32, device="cuda")
    out = torch.empty(xd.shape, dtype=torch.float64, device="cuda")
    assert _lib().amg_debug_convert(None, None, C.c_void_p(xd.data_ptr()),
                                    C.c_void_p(out.data_ptr()), xd.numel(), _stream()) == 0
    hw = xd.to(torch.float64)
    torch.cuda.synchronize()
    return out.cpu().numpy(), hw.cpu().numpy()


def _bits64(hi, lo):
    return ((hi.astype(np.uint64) << np.uint64(32)) | lo.astype(np.uint64)).view(np.float64)


def _f64_cases(rng):
    n = 1 << 20
    parts = [rng.integers(0, 2**64, n, dtype=np.uint64).view(np.float64)]  # any encoding
    # inside binary32's normal range: biased exponents 897..1150, random fraction
    e = rng.integers(897, 1151, n, dtype=np.uint64)
    s = rng.integers(0, 2, n, dtype=np.uint64)
    f = rng.integers(0, 2**52, n, dtype=np.uint64)
    parts.append(((s << np.uint64(63)) | (e << np.uint64(52)) | f).view(np.float64))
    # exact ties on the 29 dropped bits, kept fraction even and odd
    f = (rng.integers(0, 2**23, n, dtype=np.uint64) << np.uint64(29)) | np.uint64(1 << 28)
    parts.append(((s << np.uint64(63)) | (e << np.uint64(52)) | f).view(np.float64))
    # one below and one above the tie
    parts.append((((s << np.uint64(63)) | (e << np.uint64(52)) | f) - np.uint64(1)).view(np.float64))
    parts.append((((s << np.uint64(63)) | (e << np.uint64(52)) | f) + np.uint64(1)).view(np.float64))
    # exponent boundaries: the binary32 subnormal / normal edge and overflow
    for eb in (870, 873, 874, 895, 896, 897, 898, 1149, 1150, 1151, 1152):
        lo = rng.integers(0, 2**32, 4096, dtype=np.uint64)
        hi = (np.uint64(eb) << np.uint64(20)) | rng.integers(0, 2**20, 4096, dtype=np.uint64)
        parts.append(_bits64(hi, lo))
        parts.append(_bits64(hi | np.uint64(0xFFFFF), np.full(4096, 0xFFFFFFFF, np.uint64)))
        parts.append(_bits64(hi | np.uint64(0xFFFFF), np.full(4096, 0xF0000000, np.uint64)))
    fmax = float(np.finfo(np.float32).max)
    tiny = float(np.finfo(np.float32).tiny)
    special = [0.0, -0.0, np.inf, -np.inf, np.nan, -np.nan, 1.0, -1.0, fmax, -fmax,
               np.nextafter(fmax, np.inf), fmax * (1 + 2.0**-25), fmax * (1 + 2.0**-24),
               tiny, np.nextafter(tiny, 0.0), tiny / 2, 2.0**-149, 2.0**-150,
               np.nextafter(2.0**-150, 1.0), 2.0**-151, 5e-324, -5e-324, 1e308, -1e308,
               1.0 + 2.0**-24, 1.0 + 3 * 2.0**-24, 1.0 + 2.0**-24 + 2.0**-52]
    parts.append(np.array(special, np.float64))
    return np.concatenate(parts)


def test_narrowing_matches_hardware_and_ieee(amg):
    x = _f64_cases(np.random.default_rng(2406))
    got, hw = _narrow(x)
    gb, hb = got.view(np.uint32), hw.view(np.uint32)
    bad = np.flatnonzero(gb != hb)
    assert bad.size == 0, [(x[i].hex(), hex(gb[i]), hex(hb[i])) for i in bad[:8]]
    # IEEE 754 round-to-nearest-even on the host (NaN payloads aside)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32)
    ok = ~np.isnan(x)
    assert np.array_equal(gb[ok], ref.view(np.uint32)[ok])
    assert np.isnan(got[~ok]).all()


def test_widening_matches_hardware_and_ieee(amg):
    rng = np.random.default_rng(2407)
    x = rng.integers(0, 2**32, 1 << 21, dtype=np.uint64).astype(np.uint32).view(np.float32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0,
                        np.finfo(np.float32).max, np.finfo(np.float32).tiny,
                        np.float32(2.0**-149), np.float32(-(2.0**-149))], np.float32)
    x = np.concatenate([x, special])
    got, hw = _widen(x)
    gb, hb = got.view(np.uint64), hw.view(np.uint64)
    bad = np.flatnonzero(gb != hb)
    assert bad.size == 0, [(hex(x.view(np.uint32)[i]), hex(gb[i]), hex(hb[i])) for i in bad[:8]]
    ok = ~np.isnan(x)
    assert np.array_equal(gb[ok], x.astype(np.float64).view(np.uint64)[ok])


def test_convert_rejects_half_pairs(amg):
    lib = _lib()
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    assert lib.amg_debug_convert(C.c_void_p(x.data_ptr()), None, None, None, 4, _stream()) != 0
    assert lib.amg_debug_convert(None, None, None, None, -1, _stream()) != 0
    assert lib.amg_debug_convert(None, None, None, None, 0, _stream()) == 0
