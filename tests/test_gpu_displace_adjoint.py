"""The FP64 reconstruction output (recon_displace_fp64) and its adjoint
(recon_displace_adjoint, autograd.displace) against the oracle: the output
against ``oracle.displace``, the adjoint against ``oracle.displace_adjoint``
(pinned by finite differences of the oracle's forward map), and the gradient
of a loss on delta_r through the solve and the output together against the
oracle's chained adjoints."""
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


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _state(O, N, L, seed):
    b, _, _ = zeldovich_density(O, N, L, 0.8, 4.0, seed)
    t, _ = O.solve(b, L, tol=1e-12, max_cycles=60)
    return t, b


@pytest.mark.parametrize("N,L", [(16, 32.0), (24, 60.0)])
def test_displace_fp64_matches_oracle(R, O, N, L):
    t, b = _state(O, N, L, 700 + N)
    s = R.Solver(N, L)
    psi, dl = s.displace_fp64(dev(t), dev(b))
    psi_ref, dl_ref = O.displace(t, b, L)
    assert rel(psi.cpu().numpy(), psi_ref) < 1e-13
    assert np.max(np.abs(dl.cpu().numpy() - dl_ref)) < 1e-12
    s.close()


@pytest.mark.parametrize("N,L", [(16, 32.0), (24, 60.0)])
def test_displace_adjoint_matches_oracle(R, O, N, L):
    t, b = _state(O, N, L, 710 + N)
    rng = np.random.default_rng(N)
    wp = rng.standard_normal((3, N, N, N))
    wd = rng.standard_normal((N, N, N))
    s = R.Solver(N, L)
    for gp, gd in ((wp, wd), (None, wd), (wp, None)):
        gphi, gb = s.displace_adjoint(dev(t), dev(b), None if gp is None else dev(gp),
                                      None if gd is None else dev(gd))
        rt, rb = O.displace_adjoint(t, b, L, gp, gd)
        assert rel(gphi.cpu().numpy(), rt) < 1e-10
        if gd is None:
            assert not torch.any(gb)
        else:
            assert rel(gb.cpu().numpy(), rb) < 1e-10
    s.close()


def test_loss_on_delta_r_through_the_solve(R, O):
    """d/db <w, delta_r(phi(b), b)>: autograd through solve and displace vs the
    oracle's displace_adjoint followed by its solve adjoint."""
    from paper_1709_06350_gb300 import autograd
    N, L = 16, 32.0
    b, _, _ = zeldovich_density(O, N, L, 0.8, 4.0, 733)
    w = np.random.default_rng(7).standard_normal((N, N, N))
    s = R.Solver(N, L)
    bt = dev(b).requires_grad_(True)
    phi = autograd.solve(bt, s, tol=1e-13, max_cycles=60)
    _, dl = autograd.displace(phi, bt, s)
    (dl * dev(w)).sum().backward()
    t = phi.detach().cpu().numpy()
    gt, gb_direct = O.displace_adjoint(t, b, L, None, w)
    want = gb_direct + O.adjoint(t, gt, L / N)
    assert rel(bt.grad.cpu().numpy(), want) < 1e-8
    s.close()


def test_displace_adjoint_rejects_bad_arguments(R):
    N, L = 16, 32.0
    s = R.Solver(N, L)
    x = torch.ones((N,) * 3, dtype=torch.float64, device="cuda")
    out = torch.empty_like(x)
    with pytest.raises(R.ReconError):
        R.recon_displace_adjoint(s.h, N, x, x, None, x, out, out)     # outputs alias
    with pytest.raises(R.ReconError):
        R.recon_displace_adjoint(s.h, N, x, x, None, out, out, torch.empty_like(x))   # output aliases input
    # an output inside gbar_psi's 3 N^3 doubles (not at its base) overlaps it
    psi = torch.zeros((3, N, N, N), dtype=torch.float64, device="cuda")
    with pytest.raises(R.ReconError):
        R.recon_displace_adjoint(s.h, N, x, x, psi, x, psi[1], torch.empty_like(x))
    # two outputs that overlap without sharing a base address
    big = torch.empty(2 * N ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(R.ReconError):
        R.recon_displace_adjoint(s.h, N, x, x, None, x, big[:N ** 3].view(N, N, N),
                                 big[N ** 3 // 2: N ** 3 // 2 + N ** 3].view(N, N, N))
    s.close()
