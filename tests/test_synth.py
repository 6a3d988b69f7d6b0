"""The seeded input generators (no method arithmetic): the numpy backend
(oracle-side tests) and the torch backend (the bench and the GPU tests, here
on the CPU) give the same fields and particles, a seed fixes them, the field
has the requested rms, and the Zel'dovich particles sit in the box."""
import numpy as np
import pytest

from paper_1709_06350_gb300 import synth

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("N,L,sigma,seed", [(16, 32.0, 0.8, 4000), (24, 48.0, 1.0, 3000)])
def test_backends_agree(N, L, sigma, seed):
    d_np, dh_np = synth.linear_field(N, L, sigma, seed)
    d_t, dh_t = synth.linear_field(N, L, sigma, seed, backend="torch", device="cpu")
    assert np.allclose(d_t.numpy(), d_np, rtol=0, atol=1e-12 * np.abs(d_np).max())
    assert d_np.std() == pytest.approx(sigma, rel=1e-12)
    p_np = synth.zeldovich_positions(dh_np, N, L)
    p_t = synth.zeldovich_positions(dh_t, N, L).numpy()
    diff = np.abs(p_t - p_np)
    diff = np.minimum(diff, L - diff)          # a coordinate may wrap at the box edge
    assert diff.max() < 1e-9 * L
    assert p_np.shape == (N ** 3, 3) and np.all((p_np >= 0) & (p_np < L))


def test_seed_fixes_the_field():
    a, _ = synth.linear_field(16, 32.0, 1.0, 7)
    b, _ = synth.linear_field(16, 32.0, 1.0, 7)
    c, _ = synth.linear_field(16, 32.0, 1.0, 8)
    assert np.array_equal(a, b) and not np.allclose(a, c)
