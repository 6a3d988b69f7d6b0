"""The adjoint of the solve (recon_adjoint, autograd) against the oracle's
sparse-LU adjoint and against central finite differences of the GPU solve."""
import numpy as np
import pytest

from tests.workloads import zeldovich_density

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1709_06350_gb300 import build, recon
    build.build()
    return recon


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


@pytest.mark.parametrize("N,L", [(16, 32.0), (24, 48.0)])
def test_adjoint_matches_oracle(R, O, N, L):
    b, _, _ = zeldovich_density(O, N, L, 0.8, 4.0, 500 + N)
    s = R.Solver(N, L)
    phi, _ = s.solve(dev(b), tol=1e-13, max_cycles=60)
    w = np.random.default_rng(N).standard_normal((N,) * 3)
    gb = s.adjoint(dev(w)).cpu().numpy()
    ref = O.adjoint(phi.cpu().numpy(), w, L / N)
    assert abs(gb.sum()) < 1e-9 * np.abs(gb).sum()
    assert np.linalg.norm(gb - ref) < 1e-8 * np.linalg.norm(ref)
    s.close()


def test_adjoint_matches_finite_differences(R, O):
    """<w, phi(b)>: gradient vs central differences on random directions (1e-5)."""
    N, L = 32, 64.0
    b, _, _ = zeldovich_density(O, N, L, 0.8, 4.0, 77)
    bd = dev(b)
    s = R.Solver(N, L)
    w = dev(np.random.default_rng(5).standard_normal((N,) * 3))
    phi, _ = s.solve(bd, tol=1e-13, max_cycles=60)
    g = s.adjoint(w)
    rng = np.random.default_rng(6)
    eps = 1e-4
    for _ in range(4):
        d = dev(rng.standard_normal((N,) * 3))
        pp, _ = s.solve(bd + eps * d, tol=1e-13, max_cycles=60)
        lp = float((w * pp).sum())
        pm, _ = s.solve(bd - eps * d, tol=1e-13, max_cycles=60)
        lm = float((w * pm).sum())
        fd = (lp - lm) / (2 * eps)
        assert float((g * d).sum()) == pytest.approx(fd, rel=1e-5)
    s.close()


def test_autograd_solve(R, O):
    from paper_1709_06350_gb300 import autograd
    N, L = 16, 32.0
    b, _, _ = zeldovich_density(O, N, L, 0.8, 4.0, 78)
    s = R.Solver(N, L)
    bt = dev(b).requires_grad_(True)
    phi = autograd.solve(bt, s, tol=1e-13)
    loss = (phi ** 2).sum()
    loss.backward()
    ref = O.adjoint(phi.detach().cpu().numpy(), 2 * phi.detach().cpu().numpy(), L / N)
    assert np.linalg.norm(bt.grad.cpu().numpy() - ref) < 1e-8 * np.linalg.norm(ref)
    # a second solve on the same Solver invalidates the first graph node
    phi2 = autograd.solve(bt, s, tol=1e-10)
    s.solve(dev(b) * 1.01, tol=1e-10)
    with pytest.raises(RuntimeError):
        phi2.sum().backward()
    s.close()


def test_adjoint_requires_a_solve(R):
    s = R.Solver(8, 8.0)
    with pytest.raises(R.ReconError) as e:
        s.adjoint(torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda"))
    assert e.value.status == 1
    s.close()


@pytest.mark.parametrize("N,L", [(32, 64.0), (96, 192.0)])
def test_formed_and_stored_cofactors_agree(R, O, N, L):
    """The finest level's J^T with cofactors formed from phi in every
    application (the default on grids of side a multiple of 32) and with the
    six cofactor arrays kept give the same gradient up to rounding order;
    at 32^3 both also match the oracle's adjoint."""
    b, _, _ = zeldovich_density(O, N, L, 0.8, 4.0, 700 + N)
    w = np.random.default_rng(N + 1).standard_normal((N,) * 3)
    out = []
    for store in (0, 1):
        s = R.Solver(N, L, adjoint_store_cofactors=store)
        phi, _ = s.solve(dev(b), tol=1e-13, max_cycles=60)
        out.append((s.adjoint(dev(w)).cpu().numpy(), phi.cpu().numpy()))
        # a second call reuses the null vector; a changed option rebuilds it
        again = s.adjoint(dev(w)).cpu().numpy()
        assert np.linalg.norm(again - out[-1][0]) < 1e-12 * np.linalg.norm(out[-1][0])
        s.configure(adjoint_store_cofactors=1 - store)
        other = s.adjoint(dev(w)).cpu().numpy()
        assert np.linalg.norm(other - out[-1][0]) < 1e-9 * np.linalg.norm(out[-1][0])
        s.close()
    (g0, phi0), (g1, _) = out
    assert np.linalg.norm(g0 - g1) < 1e-9 * np.linalg.norm(g1)
    if N == 32:
        ref = O.adjoint(phi0, w, L / N)
        assert np.linalg.norm(g0 - ref) < 1e-8 * np.linalg.norm(ref)
