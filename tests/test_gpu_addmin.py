"""The add-min step (Table 1 MatProd followed by MatMin) on the device.

apsp_addmin_eval runs the library's own add-min form per dtype; its lane
semantics are checked against host references written from the definition:
int32 min(a + b, c); packed 16-bit per lane min((a + b) mod 2^16, c) -- the
16-bit add wraps, which is why stored values stay <= 0x7FFF; fp32
fminf(a + b, c).  apsp_addmin_peak measures the issue rate that is the
denominator of the Phase-3 roofline.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _eval(lib, dt, a, b, c):
    a_d, b_d, c_d = (torch.from_numpy(x.view(np.int32).copy()).cuda() for x in (a, b, c))
    o = torch.empty_like(a_d)
    L = lib.get_lib()
    assert L.apsp_addmin_eval(dt, ctypes.c_void_p(a_d.data_ptr()), ctypes.c_void_p(b_d.data_ptr()),
                              ctypes.c_void_p(c_d.data_ptr()), ctypes.c_void_p(o.data_ptr()), a.size, None) == 0
    torch.cuda.synchronize()
    return o.cpu().numpy().view(np.uint32)


def _words(rng, m):
    edge = np.array([0, 1, 0x7FFF, 0x7FFE, 0x8000, 0xFFFF, 0x3FFF], dtype=np.uint32)
    lo = np.concatenate([edge, rng.integers(0, 0x10000, size=m)]).astype(np.uint32)
    hi = np.concatenate([edge[::-1], rng.integers(0, 0x10000, size=m)]).astype(np.uint32)
    return lo | (hi << 16)


def test_u16x2_lanes_wrap_and_take_the_minimum(lib):
    rng = np.random.default_rng(0)
    a, b, c = _words(rng, 5000), _words(rng, 5000)[::-1].copy(), _words(rng, 5000)
    got = _eval(lib, lib.APSP_U16, a, b, c)
    for sh in (0, 16):
        la, lb, lc = ((x >> sh) & 0xFFFF for x in (a, b, c))
        exp = np.minimum((la + lb) & 0xFFFF, lc)
        np.testing.assert_array_equal((got >> sh) & 0xFFFF, exp)


def test_int32_addmin(lib):
    rng = np.random.default_rng(1)
    inf = 1073741823
    a = rng.integers(0, inf + 1, size=4096).astype(np.int64)
    b = rng.integers(0, inf + 1, size=4096).astype(np.int64)
    c = rng.integers(0, inf + 1, size=4096).astype(np.int64)
    a[:3] = [inf, 0, inf]
    b[:3] = [inf, inf, 0]
    got = _eval(lib, lib.APSP_I32, a.astype(np.uint32), b.astype(np.uint32), c.astype(np.uint32)).view(np.int32)
    np.testing.assert_array_equal(got.astype(np.int64), np.minimum(a + b, c))


def test_fp32_addmin(lib):
    rng = np.random.default_rng(2)
    a = (rng.random(4096) * 100).astype(np.float32)
    b = (rng.random(4096) * 100).astype(np.float32)
    c = (rng.random(4096) * 200).astype(np.float32)
    a[:2] = np.inf
    got = _eval(lib, lib.APSP_F32, a.view(np.uint32), b.view(np.uint32), c.view(np.uint32)).view(np.float32)
    np.testing.assert_array_equal(got, np.minimum(a + b, c))


@pytest.mark.parametrize("dt,lo,hi", [(0, 48.0, 70.0), (1, 96.0, 140.0), (2, 40.0, 140.0)])
def test_addmin_peak_per_form(lib, dt, lo, hi):
    """Relaxations per clock per SM: int32 near the SM's 64 INT32 lanes, packed 16-bit twice that, fp32 (packed pair
    add + three-input min) in between the one-add-one-min rate and twice the INT32 rate."""
    L = lib.get_lib()
    rpc, rps = ctypes.c_double(), ctypes.c_double()
    assert L.apsp_addmin_peak(0, dt, ctypes.byref(rpc), ctypes.byref(rps)) == 0
    assert lo <= rpc.value <= hi, rpc.value
    assert rps.value > 0
