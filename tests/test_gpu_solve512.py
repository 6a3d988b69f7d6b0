"""The headline workload (512^3, L = 512 Mpc/h, sigma_lin = 1, R = 2 Mpc/h)
solved on the GPU by the mixed-precision path, checked against the oracle on
sampled cells: the oracle's own determinant (Sec. II eq. basic_eqs with the
stencils of eq. discrete_examples) at 10^4 seeded random cells of the GPU's
phi gives the residual r = b + c - det(I + H phi) there, whose rms (mean
removed) over the rms of b - 1 estimates the stopping measure the GPU
reports.  A full oracle solve at 512^3 takes about ten minutes on one core;
its determinant at sampled cells takes milliseconds.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06350_gb300 import build, recon
    build.build()
    recon.load()
    return recon


def test_mixed_512_residual_on_sampled_cells(R, O):
    from paper_1709_06350_gb300 import synth
    W = synth.WORKLOADS["mixed-512"]
    N, L = W.N, W.L
    h = L / N
    dev = torch.device("cuda")
    _, dh = synth.linear_field(N, L, W.sigma_lin, W.seed, backend="torch", device=dev)
    pos = synth.zeldovich_positions(dh, N, L).contiguous()
    del dh
    s = R.Solver(N, L, R.RECON_MIXED)
    b = s.smooth_density(s.deposit_cic(pos), W.R)
    del pos
    phi, st = s.solve(b, tol=W.tol, max_cycles=40)
    assert st["rel_residual"] < W.tol
    torch.cuda.synchronize()
    phi_h = phi.cpu().numpy()
    b_h = b.cpu().numpy()
    s.close()
    rng = np.random.default_rng(512)
    ijk = rng.integers(0, N, size=(10000, 3)).astype(np.int32)
    det = O.det_cells(phi_h, h, ijk)
    bs = b_h[ijk[:, 0], ijk[:, 1], ijk[:, 2]]
    r = bs + st["compat_c"] - det
    est = np.sqrt(np.mean((r - r.mean()) ** 2)) / np.sqrt(np.mean((b_h - 1.0) ** 2))
    # the oracle's estimate of the stopping measure agrees with the GPU's to
    # sampling error (10^4 samples of a field with O(1) kurtosis: ~2%) and
    # meets the tolerance; no single sampled cell is far off
    assert est < W.tol
    assert est == pytest.approx(st["rel_residual"], rel=0.3)
    assert np.max(np.abs(r - r.mean())) < 20 * W.tol * np.sqrt(np.mean((b_h - 1.0) ** 2))
