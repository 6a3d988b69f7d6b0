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


def test_delta_r_loss_gradient_matches_finite_differences(O):
    """The full gradient of the band-limited reconstruction loss
    sum_{|k| < 0.5} |FFT(delta_r) - FFT(delta_L)|^2 with respect to the
    density b (the output's adjoint for its direct b term plus the solve's
    adjoint of its theta term) against central differences through the
    oracle's own solve, on a Zel'dovich field of the adjoint workload's
    recipe (h = 2 Mpc/h, sigma 0.8, R = 4 Mpc/h) at 16^3.  Each direction's
    step moves no q across a CIC cell face (half the largest such step, from
    the map's linear response), so the loss is smooth over it; at this size
    the step is large enough that the solves' rounding stays far below it."""
    N, L = 16, 32.0
    h = L / N
    dL, dh = synth.linear_field(N, L, 0.8, 5000)
    b = O.smooth_and_floor(O.cic_deposit(synth.zeldovich_positions(dh, N, L), N, L), L, 4.0)
    th, info = O.solve(b, L, tol=1e-14, max_cycles=80)
    assert info["status"] == 0
    kf = 2 * np.pi / L
    f = np.fft.fftfreq(N, d=1.0 / N) * kf
    fz = np.fft.rfftfreq(N, d=1.0 / N) * kf
    mask = np.sqrt(f[:, None, None] ** 2 + f[None, :, None] ** 2 + fz[None, None, :] ** 2) < 0.5
    ref = np.fft.rfftn(dL)

    def loss(dl):
        return float(np.sum(np.abs(np.fft.rfftn(dl) - ref) ** 2 * mask))

    # d loss / d delta_r: 2 Re sum over the half spectrum of mask conj(D) dD/dx
    _, dl0 = O.displace(th, b, L)
    full = np.zeros((N, N, N), dtype=complex)
    full[:, :, :N // 2 + 1] = mask * (np.fft.rfftn(dl0) - ref)
    gdl = 2.0 * N ** 3 * np.real(np.fft.ifftn(full))
    gth, gb_direct = O.displace_adjoint(th, b, L, None, gdl)
    grad = gb_direct + O.adjoint(th, gth, h)

    def ucoords(t):
        out = []
        for ax in range(3):
            g = (np.roll(t, -1, ax) - np.roll(t, 1, ax)) / (2 * h)
            shape = [1, 1, 1]
            shape[ax] = N
            x = ((np.arange(N) + 0.5) * h).reshape(shape)
            out.append(np.remainder(x + g, L) / h - 0.5)
        return out

    u0 = ucoords(th)
    dist = [np.minimum(u - np.floor(u), np.ceil(u) - u) for u in u0]

    def solve(bb):
        t, _ = O.solve(bb, L, theta0=th, tol=1e-15, max_cycles=30)
        return t

    rng = np.random.default_rng(3)
    for _ in range(3):
        d = np.fft.irfftn(np.fft.rfftn(rng.standard_normal((N, N, N))) * mask, s=(N, N, N), axes=(0, 1, 2))
        d /= np.sqrt(np.mean(d ** 2))
        e0 = 1e-7
        dphi = (solve(b + e0 * d) - solve(b - e0 * d)) / (2 * e0)
        du = [(np.roll(dphi, -1, ax) - np.roll(dphi, 1, ax)) / (2 * h * h) for ax in range(3)]
        eps = 0.5 * min(float((dist[ax] / np.maximum(np.abs(du[ax]), 1e-300)).min()) for ax in range(3))
        vals = []
        for sg in (1.0, -1.0):
            bp = b + sg * eps * d
            tp = solve(bp)
            assert all(np.all(np.floor(a) == np.floor(c)) for a, c in zip(u0, ucoords(tp)))
            vals.append(loss(O.displace(tp, bp, L)[1]))
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert float(np.sum(grad * d)) == pytest.approx(fd, rel=1e-7)
