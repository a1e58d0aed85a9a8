"""The integer arithmetic of the fixed-point passes (csrc/fxarith.cuh),
compiled for the host (tests/fxarith_host.cpp) and pinned to exact rational
arithmetic: each rounding step against its definition, ties included.

 * fx_of: a double in 55-bit fixed point relative to a binade bound `top`,
   F = round(v 2^(1077 - top)), ties to even, |F| < 2^55;
 * fx_limbs: F = hi 2^28 + lo with 0 <= lo < 2^28;
 * bitlen_u128: the bit length of a 128-bit magnitude;
 * fx_round53: the FP64 nearest to +-|v| for |v| in [2^e, 2^(e+1)) given
   by its normalised top 64 bits and a sticky bit (the residual r_j);
 * fx_round_norm: round(|v| 2^(w - e - 1)) from the same (the fixed point
   of rho_j at the CTA's exponent).
"""
import ctypes as C
import os
import shutil
import struct
import subprocess
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("fxh") / "libfxh.so")
    subprocess.run([cxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out, os.path.join(HERE, "fxarith_host.cpp")],
                   check=True)
    L = C.CDLL(out)
    L.fxh_of.argtypes = [C.c_uint64, C.c_int]
    L.fxh_of.restype = C.c_int64
    L.fxh_limbs.argtypes = [C.c_int64, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.fxh_bitlen.argtypes = [C.c_uint64, C.c_uint64]
    L.fxh_bitlen.restype = C.c_int
    L.fxh_round53.argtypes = [C.c_uint64, C.c_int, C.c_int, C.c_int]
    L.fxh_round53.restype = C.c_uint64
    L.fxh_round_norm.argtypes = [C.c_uint64, C.c_int, C.c_int]
    L.fxh_round_norm.restype = C.c_int64
    return L


def bits_of(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def double_of(b: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", b))[0]


def normalised(mag: int):
    """(Nh, Ns, L) of a positive integer: N = mag << (128 - L)."""
    L = mag.bit_length()
    N = mag << (128 - L)
    return N >> 64, int((N & ((1 << 64) - 1)) != 0), L


def random_mags(rng, count):
    """Magnitudes of every bit length 1..127, with ties and near-ties forced
    at the 53-bit and at random rounding positions."""
    out = []
    for i in range(count):
        L = int(rng.integers(1, 128))
        mag = (1 << (L - 1)) | int(rng.integers(0, 1 << 62)) << max(0, L - 63) >> max(0, 62 - L + 1)
        mag &= (1 << L) - 1
        mag |= 1 << (L - 1)
        kind = i % 4
        if kind and L > 54:
            cut = L - 53 if kind != 3 else int(rng.integers(1, L))
            base = (mag >> cut) << cut
            half = 1 << (cut - 1)
            mag = base | half if kind == 1 else (base | half | 1 if kind == 2 else base | (half - 1 if half > 1 else 0))
        out.append(mag)
    return out


def test_round53_is_correct_rounding(lib):
    rng = np.random.default_rng(1)
    for mag in random_mags(rng, 6000):
        Nh, Ns, L = normalised(mag)
        e = int(rng.integers(-1000, 1000))
        neg = int(rng.integers(0, 2))
        want = float(Fraction(mag) * Fraction(2) ** (e - L + 1))
        want = -want if neg else want
        assert lib.fxh_round53(Nh, Ns, neg, e) == bits_of(want), (mag, e, neg)


def test_round_norm_is_round_half_even(lib):
    rng = np.random.default_rng(2)
    for mag in random_mags(rng, 6000):
        Nh, Ns, L = normalised(mag)
        w = int(rng.integers(-3, 56))
        want = round(Fraction(mag) * Fraction(2) ** (w - L))        # ties to even
        assert lib.fxh_round_norm(Nh, Ns, w) == want, (mag, w)
    # exact ties at the rounding position of w: to even, either way
    for _ in range(3000):
        L = int(rng.integers(3, 128))
        w = int(rng.integers(1, min(L, 56)))
        cut = L - w
        mag = (1 << (L - 1)) | ((int(rng.integers(0, 1 << 62)) << cut) & ((1 << (L - 1)) - 1))
        mag = (mag >> cut << cut) | (1 << (cut - 1))
        Nh, Ns, L2 = normalised(mag)
        assert L2 == L
        q = mag >> cut
        assert lib.fxh_round_norm(Nh, Ns, w) == (q if q % 2 == 0 else q + 1), (mag, w)
    # the exact half at w = 0 rounds to 0, just above it to 1
    assert lib.fxh_round_norm(1 << 63, 0, 0) == 0
    assert lib.fxh_round_norm(1 << 63, 1, 0) == 1


def test_fixed_point_of_a_double(lib):
    rng = np.random.default_rng(3)
    vals = list(rng.standard_normal(2000) * np.exp(rng.uniform(-700, 700, 2000)))
    vals += [0.0, -0.0, 5e-324, -2.5e-320, 2.2250738585072014e-308, 1.7976931348623157e308, 1.0, -1.5, 3.0]
    for v in vals:
        b = bits_of(float(v))
        e = (b >> 52) & 0x7FF
        be = max(e, 1)
        for top in (be, be + 1, be + 2, be + int(rng.integers(3, 70))):
            if top > 2046:
                continue
            F = lib.fxh_of(b, top)
            want = round(Fraction(float(v)) * Fraction(2) ** (1077 - top))
            assert F == want, (v, top, F, want)
            assert abs(F) < 1 << 55
            lo, hi = C.c_int(), C.c_int()
            lib.fxh_limbs(F, C.byref(lo), C.byref(hi))
            assert 0 <= lo.value < 1 << 28 and hi.value * (1 << 28) + lo.value == F


def test_bitlen(lib):
    rng = np.random.default_rng(4)
    for _ in range(2000):
        L = int(rng.integers(1, 129))
        v = (1 << (L - 1)) | (int(rng.integers(0, 1 << 63)) % (1 << (L - 1)) if L > 1 else 0)
        assert lib.fxh_bitlen(v >> 64, v & ((1 << 64) - 1)) == L
