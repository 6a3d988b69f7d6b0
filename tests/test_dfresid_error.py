"""Error of the mixed path's double-float residual (dfresid.cuh, the
arithmetic of k_residual_df) against r = b + c - det(I + H phi) evaluated in
long double from the same phi_hi + phi_lo, on seeded potentials with the
magnitudes of the 512^3 workload (|phi|/h^2 in the hundreds, which is where
the second differences cancel).  A host program compiled from the library's
header evaluates the cell function; b is set to det - c plus a residual of
1e-9 (the converged regime, where r is all cancellation) or 0.1.

The bound: the final float rounding of r plus 32 units of 2^-48 times
max|phi|/h^2 times max(1, |det|) (the entries' absolute error, amplified by
the cofactors).  The same residual in generic double-float arithmetic
(dfloat.cuh's df_add / df_mul throughout) is evaluated beside it, and the
new error may not exceed four times the generic one plus that bound's
rounding floor."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1709_06350_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <vector>
#include "dfresid.cuh"
using namespace recon;
struct NB { float c, xp, xm, yp, ym, zp, zm, xpyp, xmym, xmyp, xpym, ypzp, ymzm, ymzp, ypzm, xpzp, xmzm, xmzp, xpzm; };
typedef long double LD;
// the same residual with generic double-float operations
static float generic(const NB &H, const NB &L, float bh, float bl, df c, df ih2)
{
    const df q4 = df_scale2(ih2, 0.25f), one = df_make(1.0f, 0.0f), C2 = df_make(2.0f * H.c, 2.0f * L.c);
    auto d2 = [&](float ph, float pl, float mh, float ml) {
        return df_add(one, df_mul(df_sub(df_add(df_make(ph, pl), df_make(mh, ml)), C2), ih2));
    };
    auto x4 = [&](float a, float al, float b, float bl_, float cc, float cl, float d, float dl) {
        return df_mul(df_sub(df_add(df_make(a, al), df_make(b, bl_)), df_add(df_make(cc, cl), df_make(d, dl))), q4);
    };
    const df xx = d2(H.xp, L.xp, H.xm, L.xm), yy = d2(H.yp, L.yp, H.ym, L.ym), zz = d2(H.zp, L.zp, H.zm, L.zm);
    const df xy = x4(H.xpyp, L.xpyp, H.xmym, L.xmym, H.xmyp, L.xmyp, H.xpym, L.xpym);
    const df yz = x4(H.ypzp, L.ypzp, H.ymzm, L.ymzm, H.ymzp, L.ymzp, H.ypzm, L.ypzm);
    const df xz = x4(H.xpzp, L.xpzp, H.xmzm, L.xmzm, H.xmzp, L.xmzp, H.xpzm, L.xpzm);
    const df det = df_add(df_sub(df_mul(xx, df_sub(df_mul(yy, zz), df_mul(yz, yz))),
                                 df_mul(xy, df_sub(df_mul(xy, zz), df_mul(yz, xz)))),
                          df_mul(xz, df_sub(df_mul(xy, yz), df_mul(yy, xz))));
    const df r = df_sub(df_add(df_make(bh, bl), c), det);
    return r.hi + r.lo;
}
int main(int argc, char **argv)
{
    const int N = atoi(argv[1]);
    const double h = atof(argv[2]), amp = atof(argv[3]), cval = atof(argv[4]);
    std::vector<double> phi((size_t)N * N * N);
    if (fread(phi.data(), 8, phi.size(), stdin) != phi.size()) return 1;
    std::vector<float> hi(phi.size()), lo(phi.size());
    for (size_t i = 0; i < phi.size(); ++i) { hi[i] = (float)phi[i]; lo[i] = (float)(phi[i] - (double)hi[i]); }
    const double ih2d = 1.0 / (h * h);
    const df ih2 = df_from_double(ih2d), c = df_from_double(cval);
    int ex;
    const bool pow2 = ih2.lo == 0.0f && std::frexp(ih2d, &ex) == 0.5;
    auto at = [&](int i, int j, int k) { return (size_t)(((i + N) % N) * N + ((j + N) % N)) * N + ((k + N) % N); };
    double err_new = 0, err_gen = 0, scale = 0, dmax = 1;
    for (int i = 0; i < N; ++i) for (int j = 0; j < N; ++j) for (int k = 0; k < N; ++k) {
        const size_t o[19] = {at(i,j,k), at(i+1,j,k), at(i-1,j,k), at(i,j+1,k), at(i,j-1,k), at(i,j,k+1), at(i,j,k-1),
                              at(i+1,j+1,k), at(i-1,j-1,k), at(i-1,j+1,k), at(i+1,j-1,k),
                              at(i,j+1,k+1), at(i,j-1,k-1), at(i,j-1,k+1), at(i,j+1,k-1),
                              at(i+1,j,k+1), at(i-1,j,k-1), at(i-1,j,k+1), at(i+1,j,k-1)};
        NB H, L; float *ph = &H.c, *pl = &L.c; LD P[19];
        for (int t = 0; t < 19; ++t) { ph[t] = hi[o[t]]; pl[t] = lo[o[t]]; P[t] = (LD)hi[o[t]] + (LD)lo[o[t]]; }
        const LD ih = (LD)ih2.hi + (LD)ih2.lo;
        const LD xx = 1 + (P[1] + P[2] - 2 * P[0]) * ih, yy = 1 + (P[3] + P[4] - 2 * P[0]) * ih;
        const LD zz = 1 + (P[5] + P[6] - 2 * P[0]) * ih;
        const LD xy = (P[7] + P[8] - P[9] - P[10]) * ih / 4, yz = (P[11] + P[12] - P[13] - P[14]) * ih / 4;
        const LD xz = (P[15] + P[16] - P[17] - P[18]) * ih / 4;
        const LD det = xx * (yy * zz - yz * yz) - xy * (xy * zz - yz * xz) + xz * (xy * yz - yy * xz);
        const LD cl = (LD)c.hi + (LD)c.lo;
        const df b = df_from_double((double)(det - cl) + amp * std::sin(0.37 * (double)o[0]));
        const LD r = (LD)b.hi + (LD)b.lo + cl - det;
        const float rn = pow2 ? dfr_residual<true>(H, L, b.hi, b.lo, c, ih2) : dfr_residual<false>(H, L, b.hi, b.lo, c, ih2);
        const float rg = generic(H, L, b.hi, b.lo, c, ih2);
        const double fl = std::fabs((double)r) * std::ldexp(1.0, -24);
        err_new = std::fmax(err_new, std::fabs((double)((LD)rn - r)) - fl);
        err_gen = std::fmax(err_gen, std::fabs((double)((LD)rg - r)) - fl);
        scale = std::fmax(scale, std::fabs(phi[o[0]]) * ih2d);
        dmax = std::fmax(dmax, std::fabs((double)det));
    }
    printf("%d %.17g %.17g %.17g %.17g\n", (int)pow2, err_new, err_gen, scale, dmax);
    return 0;
}
"""


@pytest.fixture(scope="module")
def program(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("dfresid")
    src = d / "dfresid.cu"
    src.write_text(PROGRAM)
    exe = d / "dfresid"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-Xcompiler", "-ffp-contract=off",
                    "-I" + os.path.join(ROOT, "paper_1709_06350_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    return str(exe)


def _potential(N, h, seed, big):
    """theta with del^2 theta = delta (linear order) of a seeded field, plus
    an offset of ``big`` h^2 (the magnitude the 512 Mpc/h box's longest modes
    give phi at h = 1, where their curvature is small: at this N a mode that
    large would not be) and a mild box-scale mode."""
    L = N * h
    _, dh = synth.linear_field(N, L, 1.0, seed)
    kx, ky, kz = synth._kgrid(N, L)
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    th = np.fft.irfftn(-dh / k2, s=(N, N, N), axes=(0, 1, 2))
    x = np.arange(N) * (2 * np.pi / N)
    th = th + big * h * h + 3.0 * h * h * (np.cos(x)[:, None, None] + 0.7 * np.sin(x)[None, :, None]
                                          + 0.4 * np.cos(x + 1.0)[None, None, :])
    return np.ascontiguousarray(th, dtype=np.float64)


@pytest.mark.parametrize("N,h,amp,big,c", [
    (32, 1.0, 1e-9, 600.0, 1.25e-3),      # 512^3-like magnitudes, converged regime
    (32, 1.0, 0.1, 600.0, -3e-4),         # large residual
    (32, 2.34375, 1e-9, 80.0, 2e-3),      # 1/h^2 not a power of two
    (24, 0.5, 1e-9, 2000.0, 0.0),         # 1/h^2 = 4
])
def test_residual_error_bound(program, N, h, amp, big, c):
    phi = _potential(N, h, 11 + N, big)
    out = subprocess.run([program, str(N), repr(h), repr(amp), repr(c)], input=phi.tobytes(),
                         capture_output=True, check=True).stdout.decode().split()
    pow2, err_new, err_gen, scale, dmax = int(out[0]), *map(float, out[1:])
    assert pow2 == (h in (1.0, 0.5))
    unit = 2.0 ** -48 * scale * dmax
    assert scale > 50.0      # the cancellation regime is exercised
    assert err_new <= 32 * unit, (err_new, unit)
    assert err_new <= 4 * err_gen + unit, (err_new, err_gen)
