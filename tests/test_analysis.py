import numpy as np

from paper_1709_06350_gb300 import analysis, synth


def test_correlation_limits():
    N, L = 32, 64.0
    d, _ = synth.linear_field(N, L, 1.0, 3)
    noise = np.random.default_rng(1).standard_normal((N,) * 3)
    k, r, m = analysis.correlation(d, d, L)
    assert np.allclose(r[np.isfinite(r)], 1.0)
    k, r, m = analysis.correlation(d, -2.0 * d, L)
    assert np.allclose(r[np.isfinite(r)], -1.0)
    k, r, m = analysis.correlation(d, noise, L)
    assert np.nanmax(np.abs(r[4:])) < 0.3
    # half-plane weights reproduce the shell counts of the full FFT grid
    f = np.fft.fftfreq(N, 1.0 / N)
    kk = np.sqrt(f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2)
    full = np.bincount(np.rint(kk).astype(int).ravel(), minlength=N)[:m.size]
    assert np.array_equal(m, full)


def test_correlation_torch_matches_numpy():
    torch = __import__("pytest").importorskip("torch")
    N, L = 16, 32.0
    a, _ = synth.linear_field(N, L, 1.0, 5)
    b = a + 0.5 * np.random.default_rng(2).standard_normal((N,) * 3)
    k1, r1, m1 = analysis.correlation(a, b, L)
    k2, r2, m2 = analysis.correlation(torch.from_numpy(a), torch.from_numpy(b), L)
    good = np.isfinite(r1)
    assert np.allclose(r1[good], r2[good]) and np.allclose(m1, m2)
