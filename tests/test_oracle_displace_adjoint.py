"""The oracle's adjoint of the reconstruction output (Sec. II.B as restated in
``oracle.displace``), pinned by central finite differences of the oracle's C
forward map: for L = <w_psi, psi> + <w_dl, delta_r>,
dL(theta + e dt, b + e db)/de = <gbar_theta, dt> + <gbar_b, db>.  The map is
piecewise smooth (CIC weights are linear within a cell), so the step is
small enough that no particle's q crosses a cell face."""
import numpy as np
import pytest

from paper_1709_06350_gb300 import synth


def _inputs(N, L, seed):
    h = L / N
    t = synth.smooth_field(N, seed, 0.3 * h * h, kmax=2)
    b = 1.0 + synth.smooth_field(N, seed + 1, 0.3, kmax=2)
    return t, b / b.mean()


def _loss(O, t, b, L, wp, wd):
    psi, dl = O.displace(t, b, L)
    return float(np.sum(wp * psi) + np.sum(wd * dl))


@pytest.mark.parametrize("N,L,seed", [(8, 8.0, 3), (12, 30.0, 7)])
def test_displace_adjoint_matches_finite_differences(O, N, L, seed):
    t, b = _inputs(N, L, seed)
    rng = np.random.default_rng(seed + 10)
    wp = rng.standard_normal((3, N, N, N))
    wd = rng.standard_normal((N, N, N))
    gt, gb = O.displace_adjoint(t, b, L, wp, wd)
    h = L / N
    for _ in range(6):
        dt = rng.standard_normal((N, N, N)) * h * h
        db = rng.standard_normal((N, N, N))
        eps = 1e-7   # small enough that no particle's q crosses a CIC cell face
        fd = (_loss(O, t + eps * dt, b + eps * db, L, wp, wd)
              - _loss(O, t - eps * dt, b - eps * db, L, wp, wd)) / (2 * eps)
        ad = float(np.sum(gt * dt) + np.sum(gb * db))
        assert abs(ad - fd) <= 1e-6 * max(abs(fd), 1e-3), (ad, fd)


def test_displace_adjoint_parts(O):
    """psi alone gives no gradient on b, and its theta-gradient is the
    transpose of -grad: sum_d D_d(gbar_psi_d) for central differences."""
    N, L = 8, 8.0
    t, b = _inputs(N, L, 5)
    rng = np.random.default_rng(6)
    wp = rng.standard_normal((3, N, N, N))
    gt, gb = O.displace_adjoint(t, b, L, gbar_psi=wp)
    assert np.all(gb == 0.0)
    h = L / N
    want = sum((np.roll(wp[a], -1, a) - np.roll(wp[a], 1, a)) / (2 * h) for a in range(3))
    assert np.allclose(gt, want, rtol=0, atol=1e-12 * np.abs(want).max())
    z_t, z_b = O.displace_adjoint(t, b, L)
    assert not np.any(z_t) and not np.any(z_b)
