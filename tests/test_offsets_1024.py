"""Host-side checks of the library's 32-bit grid offsets at the largest grid
it accepts (N = 1024, the 1024^3 workload): a host program compiled from the
library's own header evaluates offs(N, i, j, k) at the corners of the grid
and at random cells and compares them with 64-bit arithmetic; the component
arrays (psi, cofactor and adjoint fields) are indexed c * N^3 + offs in
64-bit, so only offs itself must fit 32 bits."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include "common.cuh"
int main(int argc, char **argv)
{
    const int N = atoi(argv[1]);
    int i, j, k;
    while (scanf("%d %d %d", &i, &j, &k) == 3) printf("%u\n", recon::offs(N, i, j, k));
    printf("maxN %d\n", recon::kMaxN);
    return 0;
}
"""


def test_offsets_at_1024(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "offs.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "offs"
    subprocess.run([nvcc, "-std=c++17", "-I" + os.path.join(ROOT, "include"),
                    "-I" + os.path.join(ROOT, "paper_1709_06350_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    N = 1024
    rng = np.random.default_rng(1024)
    cells = np.concatenate([np.array([[0, 0, 0], [N - 1, N - 1, N - 1], [N - 1, 0, 0], [0, N - 1, N - 1]]),
                            rng.integers(0, N, size=(2000, 3))])
    out = subprocess.run([str(exe), str(N)], input="\n".join(" ".join(map(str, c)) for c in cells),
                         capture_output=True, text=True, check=True).stdout.split("\n")
    got = np.array([int(x) for x in out[:len(cells)]], dtype=np.int64)
    ref = (cells[:, 0].astype(np.int64) * N + cells[:, 1]) * N + cells[:, 2]
    assert np.array_equal(got, ref)
    assert got.max() == N ** 3 - 1 < 2 ** 32
    assert out[len(cells)] == "maxN 1024"
    # the largest component index used (psi's third component, the adjoint's
    # ninth field) exceeds 32 bits only in 64-bit arithmetic
    assert 8 * N ** 3 + got.max() >= 2 ** 32
