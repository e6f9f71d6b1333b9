"""The FP32 direction maps of the walk kernel, checked on the host over every
23-bit window (no GPU): the angle pi (2u - 1) is formed as one FMA on the
bit-built float f (2-D: f = 2 + 2u, angle = f pi - 3 pi; 3-D: f = 1 + u,
angle = f 2 pi - 3 pi).  An FMA rounds once, and f times a float constant
is exact in FP64 (24 + 24 bits), so FP64 arithmetic followed by one
rounding to FP32 reproduces it exactly.  The claims of the kernel's
comments: every angle lies in [-pi, pi] (the range of the SFU sine's
documented error bound) and within 4.5e-7 rad of the exact pi (2u - 1); the
3-D z = 3 - 2 f is 1 - 2u exactly.  The constants are read from the
header, so the test follows the code."""
import re
from pathlib import Path

import numpy as np

HDR = Path(__file__).resolve().parents[1] / "paper_2409_03686_gb300" / "csrc" / "wos_device.cuh"


def _consts():
    src = HDR.read_text()
    m2 = re.search(r"__sincosf\(fmaf\(f, ([0-9.]+)f, (-[0-9.]+)f\)", src)
    m3 = re.search(r"__sincosf\(fmaf\(f2, ([0-9.]+)f, (-[0-9.]+)f\)", src)
    assert m2 and m3, "the FMA angle forms were not found in wos_device.cuh"
    return [tuple(np.float32(float(g)) for g in m.groups()) for m in (m2, m3)]


def _fma32(a, b, c):
    """fmaf(a, b, c) for float32 arrays: the FP64 value is exact here."""
    return (a.astype(np.float64) * np.float64(b) + np.float64(c)).astype(np.float32)


WIN = np.arange(1 << 23, dtype=np.uint32)


def test_2d_angle_in_range_and_close():
    (pi_f, c), _ = _consts()
    f = (np.uint32(0x40000000) | WIN).view(np.float32)  # 2 + window 2^-22
    ang = _fma32(f, pi_f, c).astype(np.float64)
    u = WIN.astype(np.float64) * 2.0 ** -23
    exact = np.pi * (2 * u - 1)
    assert ang.min() >= -np.pi and ang.max() <= np.pi
    assert np.abs(ang - exact).max() < 4.5e-7
    # the map keeps the windows' order: a sampled uniform angle stays uniform
    assert (np.diff(ang) >= 0).all()


def test_3d_angle_and_z():
    _, (two_pi_f, c) = _consts()
    f = (np.uint32(0x3f800000) | WIN).view(np.float32)  # 1 + window 2^-23
    ang = _fma32(f, two_pi_f, c).astype(np.float64)
    u = WIN.astype(np.float64) * 2.0 ** -23
    exact = np.pi * (2 * u - 1)
    assert ang.min() >= -np.pi and ang.max() <= np.pi
    assert np.abs(ang - exact).max() < 4.5e-7
    z = _fma32(f, np.float32(-2.0), np.float32(3.0)).astype(np.float64)
    np.testing.assert_array_equal(z, 1 - 2 * u)
