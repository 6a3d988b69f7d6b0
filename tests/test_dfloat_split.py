"""The double -> double-float split done with integer operations
(df_from_double_bits, used by the mixed path's split kernel) against the
FP64 definition hi = RN(x), lo = RN(x - hi) (df_from_double): bit for bit,
on random values over the whole double range and on the cases the integer
rounding has to get right (ties to even, a carry into the exponent, signs,
zero remainders, the range edges).  A host program compiled from the
library's header evaluates both.  Likewise the float -> double widening
from the bit pattern (df_f2d_bits) against the conversion instruction."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <cstring>
#include "dfloat.cuh"
int main()
{
    unsigned long long u;
    long bad = 0, n = 0;
    while (scanf("%llx", &u) == 1) {
        double x;
        std::memcpy(&x, &u, 8);
        const recon::df a = recon::df_from_double(x), b = recon::df_from_double_bits(x);
        unsigned ah, al, bh, bl;
        std::memcpy(&ah, &a.hi, 4); std::memcpy(&al, &a.lo, 4);
        std::memcpy(&bh, &b.hi, 4); std::memcpy(&bl, &b.lo, 4);
        ++n;
        if (ah != bh || al != bl) {
            if (bad < 5) printf("mismatch %016llx: %08x %08x vs %08x %08x\n", u, ah, al, bh, bl);
            ++bad;
        }
    }
    printf("checked %ld bad %ld\n", n, bad);
    return 0;
}
"""


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def test_integer_split_equals_fp64_split(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "split.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "split"
    subprocess.run([nvcc, "-std=c++17", "-Xcompiler", "-ffp-contract=off",
                    "-I" + os.path.join(ROOT, "paper_1709_06350_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    rng = np.random.default_rng(7)
    vals = []
    # random doubles of every magnitude the solver meets and beyond
    for lo, hi in [(-45, -38), (-38, -1), (-1, 3), (3, 40), (40, 126), (126, 130), (-300, -45)]:
        e = rng.uniform(lo, hi, 4000)
        vals += (rng.choice([-1.0, 1.0], 4000) * 2.0 ** e).tolist()
    words = [_bits(v) for v in vals]
    # constructed cases: exact ties (dropped bits = 2^28) with even and odd
    # kept bits, all-ones kept bits (the rounding carries into the exponent),
    # zero remainders, and the edges of the integer path's range
    for e in (1023 - 40, 1023 - 39, 1000, 1023, 1050, 1023 + 125, 1023 + 126):
        for keep in (0, 1, 2, 0x7FFFFE, 0x7FFFFF):
            for r in (0, 1, 0x0FFFFFFF, 0x10000000, 0x10000001, 0x1FFFFFFF):
                for sgn in (0, 1):
                    words.append((sgn << 63) | (e << 52) | (keep << 29) | r)
    words += [0, 1 << 63, 0x7FF0000000000000, 0xFFF0000000000000, 0x7FF8000000000000, 1]
    out = subprocess.run([str(exe)], input="\n".join("%x" % w for w in words),
                         capture_output=True, text=True, check=True).stdout
    assert out.strip().endswith("checked %d bad 0" % len(words)), out[-2000:]


WIDEN = r"""
#include <cstdio>
#include <cstring>
#include <cmath>
#include "dfloat.cuh"
int main()
{
    unsigned u;
    long bad = 0, n = 0;
    while (scanf("%x", &u) == 1) {
        float f;
        std::memcpy(&f, &u, 4);
        const double a = (double)f, b = recon::df_f2d_bits(f);
        unsigned long long ua, ub;
        std::memcpy(&ua, &a, 8); std::memcpy(&ub, &b, 8);
        ++n;
        if (ua != ub && !(std::isnan(a) && std::isnan(b))) {
            if (bad < 5) printf("mismatch %08x: %016llx vs %016llx\n", u, ua, ub);
            ++bad;
        }
    }
    printf("checked %ld bad %ld\n", n, bad);
    return 0;
}
"""


def test_integer_widening_equals_conversion(tmp_path):
    """df_f2d_bits (the widening the mixed path's final conversion uses)
    equals the float -> double conversion bit for bit: random patterns over
    every exponent, signed zeros, subnormals, the normal range's edges,
    infinities and NaNs."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "widen.cu"
    src.write_text(WIDEN)
    exe = tmp_path / "widen"
    subprocess.run([nvcc, "-std=c++17", "-Xcompiler", "-ffp-contract=off",
                    "-I" + os.path.join(ROOT, "paper_1709_06350_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    rng = np.random.default_rng(11)
    words = rng.integers(0, 2 ** 32, 40000, dtype=np.uint64).tolist()
    for e in (0, 1, 2, 126, 127, 128, 253, 254, 255):
        for m in (0, 1, 2, 0x400000, 0x7FFFFE, 0x7FFFFF):
            for sgn in (0, 1):
                words.append((sgn << 31) | (e << 23) | m)
    out = subprocess.run([str(exe)], input="\n".join("%x" % w for w in words),
                         capture_output=True, text=True, check=True).stdout
    assert out.strip().endswith("checked %d bad 0" % len(words)), out[-2000:]
