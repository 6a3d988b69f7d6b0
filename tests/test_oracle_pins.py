"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these re-types the oracle's own formula: each compares it with a
closed form, an identity, the paper's appendix stencils, a textbook
definition or a brute-force solve.  ``test_mutations_are_caught`` plants
plausible mistakes in a copy of the oracle and checks that a pin fails.
"""
import numpy as np
import pytest

from paper_1709_06350_gb300 import synth


def roll(a, di=0, dj=0, dk=0):
    """a[i+di, j+dj, k+dk] with periodic wrap."""
    return np.roll(a, shift=(-di, -dj, -dk), axis=(0, 1, 2))


# --------------------------------------------------------------- the cubic
@pytest.mark.parametrize("a,s_expected", [(-0.9, 2.1), (0.0, 3.0), (3.0, 6.0),
                                          (4.0, 7.0), (10.0, 13.0)])
def test_plane_cubic_worked_values(O, a, s_expected):
    """Plane case H = diag(a,0,0): p = -3a^2, q = 2a^3 - 27(1+a), root 3 + a.

    a = 4 is where the printed Delta<0 formula of eq. root fails (it gives
    3.43); a = 3 is the Delta = 0 transition with a double root at -3.
    """
    p, q = -3 * a * a, 2 * a ** 3 - 27 * (1 + a)
    assert O.largest_root(p, q) == pytest.approx(s_expected, abs=1e-12)


def test_printed_root_formula_is_not_the_physical_root():
    """The Delta<0 branch exactly as printed in eq. root, for a = 4: not a root."""
    a = 4.0
    p, q = -3 * a * a, 2 * a ** 3 - 27 * (1 + a)
    sigma = np.arccos(np.clip((3 * q / (2 * p)) * np.sqrt(-3 / p), -1, 1))
    printed = 3.0 + (-3.0 - np.sqrt(-p / 3) * np.cos((sigma + 2 * np.pi) / 3))
    assert abs(printed ** 3 + p * printed + q) > 1.0


def test_largest_root_vs_numpy_roots(O):
    rng = np.random.default_rng(7)
    for _ in range(400):
        p = -abs(rng.normal()) * 10 ** rng.uniform(-8, 2)
        q = rng.normal() * 10 ** rng.uniform(-2, 2)
        roots = np.roots([1.0, 0.0, p, q])
        ref = max(r.real for r in roots if abs(r.imag) < 1e-7 * max(1, abs(r)))
        got = O.largest_root(p, q)
        assert abs(got - ref) <= 1e-8 * max(1.0, abs(ref))
        assert abs(got ** 3 + p * got + q) <= 1e-9 * max(1.0, abs(q), abs(p * got))


def test_root_small_p_no_cancellation(O):
    """Near delta = 0 (p -> 0) the cancellation-free Cardano form stays exact."""
    for rhs in (0.5, 1.0, 1.7):
        for p in (-1e-12, -1e-9, -1e-6):
            q = -27 * rhs
            s = O.largest_root(p, q)
            assert abs(s ** 3 + p * s + q) < 1e-12 * 27 * rhs


# --------------------------------------------------------------- identities
def _theta(N, seed, amp):
    return synth.smooth_field(N, seed, amp, kmax=3) + 1e-3 * np.random.default_rng(
        seed).standard_normal((N,) * 3)


def test_cubic_is_27_det(O):
    """27 det(I + H) = s^3 + p s + 27 det(Hbar): with rhs = det(I+H) the cubic
    of eq. final_PDE vanishes at the current s (two independent oracle paths:
    the 3x3 determinant and the trace/traceless split)."""
    N, h = 8, 0.7
    t = _theta(N, 1, 0.05)
    det = O.det_grid(t, h)
    s, p, q = O.cubic_grid(t, det, 0.0, h)
    f = s ** 3 + p * s + q
    assert np.max(np.abs(f)) < 1e-12 * 27


def _appendix_sums(t, h):
    X = roll(t, 1) + roll(t, -1)
    Y = roll(t, 0, 1) + roll(t, 0, -1)
    Z = roll(t, 0, 0, 1) + roll(t, 0, 0, -1)
    Exy = roll(t, 1, 1) + roll(t, -1, -1) - roll(t, 1, -1) - roll(t, -1, 1)
    Exz = roll(t, 1, 0, 1) + roll(t, -1, 0, -1) - roll(t, 1, 0, -1) - roll(t, -1, 0, 1)
    Eyz = roll(t, 0, 1, 1) + roll(t, 0, -1, -1) - roll(t, 0, -1, 1) - roll(t, 0, 1, -1)
    return X, Y, Z, Exy, Exz, Eyz


def _appendix_A1(t, h):
    """Appendix, first stencil (tr Hbar^2), transcribed term by term."""
    X, Y, Z, Exy, Exz, Eyz = _appendix_sums(t, h)
    return ((X + Y - 2 * Z) ** 2 + (Y + Z - 2 * X) ** 2 + (Z + X - 2 * Y) ** 2) / (9 * h ** 4) \
        + (Exy ** 2 + Exz ** 2 + Eyz ** 2) / (8 * h ** 4)


def _appendix_A2(t, h, fixed=True):
    """Appendix, second stencil (tr Hbar^3).  The third 1/16 term is printed
    with the xy-edge combination; ``fixed`` uses the yz edge instead."""
    X, Y, Z, Exy, Exz, Eyz = _appendix_sums(t, h)
    h6 = h ** 6
    v = (X * (2 * X ** 2 + Y ** 2 + Z ** 2) + Y * (2 * Y ** 2 + Z ** 2 + X ** 2)
         + Z * (2 * Z ** 2 + X ** 2 + Y ** 2)) / (9 * h6)
    v -= 2 * (X ** 2 * (Y + Z) + Y ** 2 * (Z + X) + Z ** 2 * (X + Y)) / (9 * h6)
    v -= 2 * (X * (Y - Z) ** 2 + Y * (Z - X) ** 2 + Z * (X - Y) ** 2) / (9 * h6)
    v += (X + Y - 2 * Z) * Exy ** 2 / (16 * h6)
    v += (Z + X - 2 * Y) * Exz ** 2 / (16 * h6)
    v += (Y + Z - 2 * X) * (Eyz if fixed else Exy) ** 2 / (16 * h6)
    v += 3 * Exy * Exz * Eyz / (32 * h6)
    return v


def test_appendix_A1_equals_oracle_p(O):
    N, h = 8, 1.3
    t = _theta(N, 2, 0.8)
    _, p, _ = O.cubic_grid(t, np.zeros_like(t), 0.0, h)
    A1 = _appendix_A1(t, h)
    assert np.allclose(p, -4.5 * A1, rtol=1e-12, atol=1e-13 * np.abs(p).max())


def test_appendix_A2_fixed_equals_oracle_q(O):
    N, h = 8, 1.3
    t = _theta(N, 3, 0.8)
    g = np.random.default_rng(0).uniform(0.5, 2.0, (N,) * 3)
    _, _, q = O.cubic_grid(t, g, 0.0, h)
    trHb3 = (q + 27 * g) / 9.0
    A2 = _appendix_A2(t, h, fixed=True)
    assert np.allclose(trHb3, A2, rtol=1e-10, atol=1e-12 * np.abs(A2).max())
    # the printed form differs wherever the xy and yz edge terms differ
    A2p = _appendix_A2(t, h, fixed=False)
    assert np.max(np.abs(A2p - A2)) > 1e-3 * np.abs(A2).max()


# --------------------------------------------------------------- solves
SOLVE = dict(tol=1e-12, max_cycles=40)


def test_delta_zero_gives_zero_bitwise(O):
    """P1: b == 1 => theta == 0, c == 0 exactly (p = 0, q = -27, root 3)."""
    b = np.ones((16,) * 3)
    t, info = O.solve(b, 64.0, **SOLVE)
    assert np.all(t == 0.0) and info["c"] == 0.0 and info["rel_residual"] == 0.0


def _periodic_poisson_1d(delta, h):
    """Closed form of D_xx theta = delta on a periodic line (mean-free delta)."""
    N = delta.size
    m = np.arange(N)
    lam = -4.0 * np.sin(np.pi * m / N) ** 2 / h ** 2
    dh = np.fft.fft(delta)
    th = np.zeros_like(dh)
    th[1:] = dh[1:] / lam[1:]
    return np.fft.ifft(th).real


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_plane_symmetric_closed_form(O, axis):
    """P2: theta = theta(x) makes det(I+H) = 1 + D_xx theta exactly linear.
    delta reaches > 3 so cells take the three-real-root (Delta < 0) branch."""
    N, L = 16, 40.0
    h = L / N
    x = np.arange(N) / N
    prof = 0.1 + 3.0 * np.exp(-((x - 0.4) / 0.06) ** 2) + 0.3 * np.sin(2 * np.pi * x) ** 2
    d = prof / prof.mean() - 1.0
    offset = 0.15   # mean(b) = 1.15: the compatibility scalar must absorb it
    shape = [1, 1, 1]
    shape[axis] = N
    b = np.broadcast_to((1.0 + offset + d).reshape(shape), (N,) * 3).copy()
    t, info = O.solve(b, L, **SOLVE)
    ref = _periodic_poisson_1d(d, h)
    got = t.mean(axis=tuple(a for a in range(3) if a != axis))
    assert d.max() > 3.0
    assert info["status"] == 0
    assert np.max(np.abs(got - ref)) < 1e-9 * np.max(np.abs(ref))
    assert info["c"] == pytest.approx(-offset, abs=1e-11)


def test_separable_potential(O):
    """P3: theta = f(x)+g(y)+k(z): det(I+H) = prod(1 + D_aa) exactly."""
    N, L = 16, 32.0
    h = L / N
    x = np.arange(N) / N
    f = 0.9 * np.sin(2 * np.pi * x + 0.2)
    g = 0.6 * np.cos(4 * np.pi * x) + 0.3 * np.sin(2 * np.pi * x)
    k = 0.7 * np.sin(2 * np.pi * x + 1.0) - 0.2 * np.cos(6 * np.pi * x)
    d2 = lambda u: (np.roll(u, -1) + np.roll(u, 1) - 2 * u) / h ** 2
    b = ((1 + d2(f))[:, None, None] * (1 + d2(g))[None, :, None]
         * (1 + d2(k))[None, None, :])
    th_ref = f[:, None, None] + g[None, :, None] + k[None, None, :]
    th_ref = th_ref - th_ref.mean()
    t, info = O.solve(b, L, **SOLVE)
    assert info["status"] == 0 and info["cycles"] <= 15
    assert np.max(np.abs(t - th_ref)) < 1e-9 * np.max(np.abs(th_ref))
    assert abs(info["c"]) < 1e-11


@pytest.mark.parametrize("perm", [(0, 1, 2), (1, 2, 0), (0, 2, 1)])
def test_diagonal_plane_wave(O, perm):
    """P4: theta = f(i+j) exercises the mixed (edge) stencil:
    det(I+H) = (1+A)^2 - B^2, A = D_hh f, B = (f(u+2)+f(u-2)-2f(u))/(4h^2).
    Axis permutations move the wave onto the yz and xz planes."""
    N, L = 16, 24.0
    h = L / N
    u = np.arange(2 * N)
    fu = 0.5 * np.sin(2 * np.pi * u / N) + 0.25 * np.cos(4 * np.pi * u / N + 0.4)
    F = lambda v: fu[np.mod(v, N)]
    i, j = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    U = i + j
    A = (F(U + 1) + F(U - 1) - 2 * F(U)) / h ** 2
    B = (F(U + 2) + F(U - 2) - 2 * F(U)) / (4 * h ** 2)
    b2 = (1 + A) ** 2 - B ** 2
    th2 = F(U)
    b = np.broadcast_to(b2[:, :, None], (N,) * 3).transpose(perm).copy()
    th_ref = np.broadcast_to(th2[:, :, None], (N,) * 3).transpose(perm).copy()
    th_ref -= th_ref.mean()
    t, info = O.solve(b, L, **SOLVE)
    assert info["status"] == 0
    assert np.max(np.abs(t - th_ref)) < 1e-9 * np.max(np.abs(th_ref))


def test_manufactured_sinusoids(O):
    """P5: b := det_h(I + H theta*) is compatible by construction (c* = 0)."""
    N, L = 32, 64.0
    h = L / N
    ts = synth.smooth_field(N, 11, 1.6, kmax=3)
    b = O.det_grid(ts, h)
    A = np.stack([b]).min()
    assert A > 0.1
    t, info = O.solve(b, L, **SOLVE)
    assert info["status"] == 0 and info["cycles"] <= 15
    assert np.max(np.abs(t - (ts - ts.mean()))) < 1e-9 * np.max(np.abs(ts))
    assert abs(info["c"]) < 1e-11


def test_small_delta_linear_limit(O):
    """P6: ||theta - theta_Poisson|| / ||theta|| scales like epsilon."""
    N, L = 16, 32.0
    h = L / N
    s = synth.smooth_field(N, 5, 1.0, kmax=2)
    m = np.fft.fftfreq(N, 1.0 / N)
    lam = sum(-4 * np.sin(np.pi * mm / N) ** 2 / h ** 2 for mm in np.meshgrid(m, m, m, indexing="ij"))
    lam[0, 0, 0] = 1.0
    errs = []
    for eps in (1e-3, 1e-2):
        sh = np.fft.fftn(eps * s) / lam
        sh[0, 0, 0] = 0.0
        tp = np.fft.ifftn(sh).real
        t, info = O.solve(1.0 + eps * s, L, **SOLVE)
        errs.append(np.linalg.norm(t - tp) / np.linalg.norm(t))
    slope = np.log10(errs[1] / errs[0])
    assert 0.9 < slope < 1.1


def _brute_force_newton(O, b, h):
    """Dense Newton on [det(I+H theta) - b - c = 0, mean(theta) = 0] with a
    central finite-difference Jacobian of the determinant."""
    N = b.shape[0]
    n = N ** 3
    x = np.zeros(n + 1)

    def F(x):
        t = x[:n].reshape(b.shape)
        return np.concatenate([(O.det_grid(t, h) - b - x[n]).ravel(), [x[:n].mean()]])

    for _ in range(30):
        Fx = F(x)
        if np.max(np.abs(Fx)) < 1e-14:
            break
        Jm = np.empty((n + 1, n + 1))
        eps = 1e-6
        for col in range(n + 1):
            e = np.zeros(n + 1)
            e[col] = eps
            Jm[:, col] = (F(x + e) - F(x - e)) / (2 * eps)
        x = x - np.linalg.solve(Jm, Fx)
    return x[:n].reshape(b.shape), x[n]


@pytest.mark.parametrize("N", [4, 6, 8])
def test_brute_force_dense_newton(O, N):
    """P7: the multigrid answer equals a dense Newton solve of the same
    discrete system (N = 8 exercises a two-level hierarchy)."""
    L = 2.0 * N
    h = L / N
    rng = np.random.default_rng(N)
    b = 1.0 + synth.smooth_field(N, 100 + N, 0.4, kmax=1) + 0.02 * rng.standard_normal((N,) * 3)
    t_bf, c_bf = _brute_force_newton(O, b, h)
    t, info = O.solve(b, L, tol=1e-13, max_cycles=60)
    assert info["status"] == 0
    assert np.max(np.abs(t - t_bf)) < 1e-10 * max(1e-3, np.max(np.abs(t_bf)))
    assert info["c"] == pytest.approx(c_bf, abs=1e-11)


def test_symmetries(O):
    """P8: translation, axis permutation and reflection of b carry over to theta."""
    N, L = 16, 32.0
    b = O.smooth_and_floor(1.0 + synth.smooth_field(N, 21, 0.8, kmax=2), L, 0.0)
    t, _ = O.solve(b, L, **SOLVE)
    scale = np.max(np.abs(t))
    tr, _ = O.solve(np.roll(b, (3, 5, 1), axis=(0, 1, 2)), L, **SOLVE)
    assert np.max(np.abs(tr - np.roll(t, (3, 5, 1), axis=(0, 1, 2)))) < 1e-9 * scale
    tp, _ = O.solve(b.transpose(2, 0, 1), L, **SOLVE)
    assert np.max(np.abs(tp - t.transpose(2, 0, 1))) < 1e-9 * scale
    tf, _ = O.solve(b[::-1], L, **SOLVE)
    assert np.max(np.abs(tf - t[::-1])) < 1e-9 * scale


@pytest.mark.parametrize("ordering,rule", [("rb-lex", "newton1"), ("4-colour", "newton1"),
                                           ("rb-snapshot", "exact")])
def test_orderings_reach_the_same_solution(O, ordering, rule):
    """Every ordering / update rule of the paper converges to the one theta*."""
    N, L = 16, 32.0
    b = O.smooth_and_floor(1.0 + synth.smooth_field(N, 31, 1.2, kmax=2), L, 0.0)
    t0, i0 = O.solve(b, L, **SOLVE)
    t1, i1 = O.solve(b, L, ordering=ordering, rule=rule, **SOLVE)
    assert i0["status"] == 0 and i1["status"] == 0
    assert np.max(np.abs(t1 - t0)) < 1e-9 * np.max(np.abs(t0))


def test_nested_start_reaches_the_same_solution(O):
    """The nested-iteration start (coarsest grid first) and the paper's start
    from theta = 0 on the finest grid converge to the same theta*; the nested
    start needs no more cycles."""
    N, L = 16, 32.0
    b = O.smooth_and_floor(1.0 + synth.smooth_field(N, 37, 1.0, kmax=2), L, 0.0)
    t0, i0 = O.solve(b, L, fmg=True, **SOLVE)
    t1, i1 = O.solve(b, L, theta0=np.zeros_like(b), fmg=False, **SOLVE)
    assert i0["status"] == 0 and i1["status"] == 0
    assert np.max(np.abs(t1 - t0)) < 1e-9 * np.max(np.abs(t0))
    assert i0["cycles"] <= i1["cycles"]


def test_num_levels(O):
    assert [O.num_levels(n) for n in (4, 6, 8, 32, 96, 192, 512)] == [1, 1, 2, 4, 5, 6, 8]


# --------------------------------------------------------------- transfers
def test_restriction_is_eight_son_mean(O):
    a = np.random.default_rng(3).standard_normal((8, 8, 8))
    ref = a.reshape(4, 2, 4, 2, 4, 2).mean(axis=(1, 3, 5))
    assert np.allclose(O.restrict(a), ref, rtol=0, atol=1e-15)


def test_prolongation_reproduces_linear_fields(O):
    """Trilinear cell-centred interpolation is exact on linear fields (checked
    away from the periodic seam) and adds a constant everywhere."""
    Nc = 8
    Xc = (np.arange(Nc) + 0.5) / Nc
    Xf = (np.arange(2 * Nc) + 0.5) / (2 * Nc)
    for ax in range(3):
        sh = [1, 1, 1]
        sh[ax] = Nc
        c = np.broadcast_to((3.0 * Xc - 1.0).reshape(sh), (Nc,) * 3).copy()
        out = O.prolong_add(c, np.zeros_like(c), np.zeros((2 * Nc,) * 3))
        sh[ax] = 2 * Nc
        ref = np.broadcast_to((3.0 * Xf - 1.0).reshape(sh), (2 * Nc,) * 3)
        inner = [slice(None)] * 3
        inner[ax] = slice(1, 2 * Nc - 1)
        assert np.allclose(out[tuple(inner)], ref[tuple(inner)], atol=1e-14)
    cst = O.prolong_add(np.full((4,) * 3, 2.5), np.full((4,) * 3, 0.5), np.ones((8,) * 3))
    assert np.allclose(cst, 3.0, atol=1e-15)
    assert np.allclose(O.restrict(cst), 3.0, atol=1e-15)


# --------------------------------------------------------------- CIC
def test_cic_lattice_is_uniform(O):
    N, L = 32, 64.0
    rho = O.cic_deposit(synth.lattice_positions(N, L), N, L)
    assert np.all(rho == 1.0)


def test_cic_textbook_definition(O):
    """Against W(x) = prod max(0, 1 - |x - x_cell|/h) with periodic distances."""
    N, L = 6, 9.0
    h = L / N
    rng = np.random.default_rng(4)
    pos = rng.uniform(0, L, (40, 3))
    pos[0] = [0.0, L - 1e-12, 4.5]     # seam and exact face
    pos[1] = [0.75, 2.25, 3.75]        # exact cell centres
    rho = O.cic_deposit(pos, N, L, mass=1.0)
    cen = (np.arange(N) + 0.5) * h
    ref = np.zeros((N,) * 3)
    for p in pos:
        w = []
        for d in range(3):
            dist = np.abs(p[d] - cen)
            dist = np.minimum(dist, L - dist)
            w.append(np.maximum(0.0, 1.0 - dist / h))
        ref += w[0][:, None, None] * w[1][None, :, None] * w[2][None, None, :]
    assert np.allclose(rho, ref, atol=1e-13)
    assert rho.sum() == pytest.approx(40.0, abs=1e-12)
    cells, frac = O.cic_cells(pos[1:2], N, L)
    assert np.all(frac == 0.0) and list(cells[0]) == [0, 1, 2]


# --------------------------------------------------------------- NGP / TSC
def _cardinal_bspline(order):
    """scipy's B-spline basis element of degree `order` on unit-spaced knots
    centred on 0: the box, hat and quadratic kernels of NGP, CIC and TSC."""
    from scipy.interpolate import BSpline
    knots = np.arange(order + 2) - (order + 1) / 2.0
    return BSpline.basis_element(knots, extrapolate=False)


@pytest.mark.parametrize("scheme,order", [("ngp", 0), ("cic", 1), ("tsc", 2)])
def test_assignment_is_the_cardinal_bspline(O, scheme, order):
    """One particle gives cell c the product over axes of B((c + 1/2) - x/h),
    B the cardinal B-spline of degree 0 (NGP), 1 (CIC) or 2 (TSC), with
    periodic distances (Sec. I footnote names the three schemes)."""
    N, L = 8, 12.0
    h = L / N
    B = _cardinal_bspline(order)
    rng = np.random.default_rng(17 + order)
    for x in rng.uniform(-0.3 * L, 1.3 * L, (12, 3)):
        rho = O.assign_deposit(x[None, :], N, L, scheme, mass=1.0)
        ref = np.ones((N, N, N))
        for a in range(3):
            dist = (np.arange(N) + 0.5) - x[a] / h
            dist = (dist + N / 2) % N - N / 2          # minimum image, in cells
            w = np.nan_to_num(B(dist))
            shape = [1, 1, 1]
            shape[a] = N
            ref = ref * w.reshape(shape)
        assert np.allclose(rho, ref, atol=1e-14), (scheme, x)


@pytest.mark.parametrize("scheme", ["ngp", "cic", "tsc"])
def test_assignment_lattice_and_mass(O, scheme):
    """Particles on the cell centres give exactly 1 everywhere for every
    scheme; any particle set deposits its total mass."""
    N, L = 16, 20.0
    rho = O.assign_deposit(synth.lattice_positions(N, L), N, L, scheme)
    assert np.all(rho == 1.0)
    rng = np.random.default_rng(23)
    pos = rng.uniform(-L, 2 * L, (500, 3))
    rho = O.assign_deposit(pos, N, L, scheme, mass=0.37)
    assert rho.sum() == pytest.approx(500 * 0.37, rel=1e-13)
    assert rho.min() >= 0.0


def test_convergence_insensitive_to_tracer_and_mesh(O):
    """Sec. I: with 8 N^3 particles on an N^3 mesh, or N^3 particles on an
    (2N)^3 mesh, the relaxation converges at a rate similar to the default
    N^3 on N^3 (here: FAS cycle counts to 1e-8 within two of each other, for
    NGP, CIC and TSC densities of the same seeded field)."""
    N, L, R = 16, 64.0, 8.0
    cycles = {}
    for label, n_lat, n_mesh in (("N3 on N3", N, N), ("8N3 on N3", 2 * N, N), ("N3 on 8N3", N, 2 * N)):
        _, dh = synth.linear_field(n_lat, L, 0.8, 31)
        pos = synth.zeldovich_positions(dh, n_lat, L)
        for scheme in ("ngp", "cic", "tsc"):
            b = O.smooth_and_floor(O.assign_deposit(pos, n_mesh, L, scheme), L, R)
            _, info = O.solve(b, L, tol=1e-8, max_cycles=40)
            assert info["status"] == 0, (label, scheme)
            cycles[(label, scheme)] = info["cycles"]
    assert max(cycles.values()) - min(cycles.values()) <= 2, cycles


# --------------------------------------------------------------- displacement
def test_displace_zero_and_plane(O):
    N, L = 16, 32.0
    h = L / N
    psi, dr = O.displace(np.zeros((N,) * 3), np.ones((N,) * 3), L)
    assert np.all(psi == 0.0) and np.all(dr == 0.0)
    x = np.arange(N) / N
    f = 0.8 * np.sin(2 * np.pi * x)
    t = np.broadcast_to(f[:, None, None], (N,) * 3).copy()
    b = O.det_grid(t, h)
    psi, dr = O.displace(t, b, L)
    assert np.all(psi[1] == 0.0) and np.all(psi[2] == 0.0)
    assert np.allclose(psi[0][:, 0, 0], -(np.roll(f, -1) - np.roll(f, 1)) / (2 * h), atol=1e-15)
    assert np.allclose(dr, dr[:, :1, :1], atol=1e-14)
    assert dr.max() < 3.0


def test_displace_linear_limit(O):
    """For small theta, delta_r(q) -> lap theta with an O(eps^2) remainder."""
    N, L = 16, 32.0
    h = L / N
    s = synth.smooth_field(N, 8, 1.0, kmax=2)
    errs = []
    for eps in (1e-3, 1e-2):
        t = eps * s
        lap = sum(roll(t, *d) for d in [(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
                                         (0, 0, 1), (0, 0, -1)]) - 6 * t
        lap /= h * h
        _, dr = O.displace(t, O.det_grid(t, h), L)
        errs.append(np.linalg.norm(dr - lap) / np.linalg.norm(lap))
    assert 0.85 < np.log10(errs[1] / errs[0]) < 1.15


def _plane_zeldovich(N, L, A):
    """A 1-D Zel'dovich map without shell crossing and its potential in closed
    form.  Lagrangian q moves to x = q - (A/k) sin(kq), k = 2 pi / L, so the
    linear density is delta_L(q) = -d psi/dq = A cos(kq) and, for A < 1, the
    map is monotone (no shell crossing).  Its inverse q(x) is the gradient of
    x^2/2 + theta(x) with theta' = q - x = (A/k) sin(k q(x)); integrating in q
    (dx = (1 - A cos kq) dq) gives the closed form
        theta(x) = -(A/k^2) cos(k q) + (A^2 / (4 k^2)) cos(2 k q),  q = q(x).
    q(x) solves Kepler's equation x = q - (A/k) sin(kq) (Newton, to round-off).
    Returns theta and q at the cell centres x = (i + 1/2) h."""
    k = 2.0 * np.pi / L
    x = (np.arange(N) + 0.5) * (L / N)
    q = x.copy()
    for _ in range(60):
        q -= (q - (A / k) * np.sin(k * q) - x) / (1.0 - A * np.cos(k * q))
    assert np.max(np.abs(q - (A / k) * np.sin(k * q) - x)) < 1e-12 * L
    theta = -(A / k**2) * np.cos(k * q) + (A**2 / (4.0 * k**2)) * np.cos(2.0 * k * q)
    return theta, q, x


@pytest.mark.parametrize("A", [0.3, 0.5])
def test_displace_recovers_plane_zeldovich(O, A):
    """P10 (Sec. II.B, eq. reconstructed_density; steps B2-B3): a Zel'dovich
    map without shell crossing is recovered exactly in the continuum, so the
    reconstructed density at the Lagrangian grid must converge to the seeded
    delta_L(q) = A cos(kq) and psi = x - q to the exact displacement as N
    doubles -- at O(1) amplitude, where a wrong sign of q = x + grad theta,
    a dropped mass weight in either CIC average, or a wrong sign in
    v = 3 - tr((I+H)^-1) leaves an O(A) error that does not shrink.
    A <= 0.5 keeps b <= 2, so Eulerian cells sit at most 2h apart in q and
    every Lagrangian cell receives CIC weight (at A = 0.7 some cells in the
    densest region get none)."""
    L = 100.0
    errs, perrs = [], []
    for N in (16, 32, 64):
        h = L / N
        th, q, x = _plane_zeldovich(N, L, A)
        t = np.broadcast_to(th[:, None, None], (N,) * 3).copy()
        psi, dr = O.displace(t, O.det_grid(t, h), L)
        # the map is plane-symmetric: every (j, k) column carries the same profile
        assert np.all(dr == dr[:, :1, :1]) and np.all(psi[1] == 0.0) and np.all(psi[2] == 0.0)
        qg = (np.arange(N) + 0.5) * h
        errs.append(np.sqrt(np.mean((dr[:, 0, 0] - A * np.cos(2 * np.pi * qg / L)) ** 2)))
        perrs.append(np.max(np.abs(psi[0][:, 0, 0] - (x - q))))
    assert errs[-1] < 0.02 * A
    assert errs[1] < 0.75 * errs[0] and errs[2] < 0.75 * errs[1]
    # psi is a central difference of the closed-form theta: second order
    assert 2.5 < perrs[0] / perrs[1] < 5.0 and 2.5 < perrs[1] / perrs[2] < 5.0


def test_paper_eps_plane_closed_form(O):
    """The paper's epsilon (Sec. II.A.2, eq. discretisition): rms over cells of
    lap_h theta - Sigma, Sigma = the cubic's largest root - 3.  For a plane
    theta(x) the discrete Hessian is diag(a, 0, 0), a = D_xx theta, and the
    cubic factorises: s^3 + p s + q = (s - a)^2 (s + 2a) - 27 rhs.  Choosing
    for every cell a root s* = 3 + a + d (d small, so s* > |a|, the largest
    root) and rhs = (s* - a)^2 (s* + 2a) / 27 makes L_h = -d in closed form:
    epsilon = rms(d).  The right side is split into g + c with c != 0."""
    N, L = 12, 30.0
    h = L / N
    x = np.arange(N) / N
    f = 2.0 * np.sin(2 * np.pi * x) + 0.5 * np.cos(6 * np.pi * x)
    t = np.broadcast_to(f[:, None, None], (N,) * 3).copy()
    a = (np.roll(f, -1) + np.roll(f, 1) - 2 * f) / h**2
    rng = np.random.default_rng(5)
    d = 0.05 * rng.standard_normal((N,) * 3)
    s_star = 3.0 + a[:, None, None] + d
    assert np.all(s_star > np.abs(a)[:, None, None])
    rhs = (s_star - a[:, None, None]) ** 2 * (s_star + 2 * a[:, None, None]) / 27.0
    c = 0.37
    eps = O.paper_eps(t, rhs - c, c, h)
    assert eps == pytest.approx(np.sqrt(np.mean(d**2)), rel=1e-9)
    # the exact plane solution (rhs = 1 + a) has epsilon 0 to round-off
    assert O.paper_eps(t, np.broadcast_to(1.0 + a[:, None, None], (N,) * 3) - c, c, h) < 1e-13


# --------------------------------------------------------------- density preparation
@pytest.mark.parametrize("m", [(1, 0, 0), (0, 2, 0), (1, 2, 3), (8, 0, 0), (3, -5, 8)])
def test_smoothing_window_on_single_modes(O, m):
    """The Gaussian window of width R (Sec. III) on a single Fourier mode
    cos(2 pi m.i / N): the mode is an eigenfunction of the filter with
    eigenvalue exp(-k^2 R^2 / 2), k = 2 pi |m| / L (m = 8 on N = 16 is the
    Nyquist mode), the mean stays 1 and nothing reaches the floor."""
    N, L, R = 16, 40.0, 3.0
    i, j, k = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    phase = 2.0 * np.pi * (m[0] * i + m[1] * j + m[2] * k) / N
    rho = 1.0 + 0.3 * np.cos(phase + 0.4)
    kk = 2.0 * np.pi * np.sqrt(m[0] ** 2 + m[1] ** 2 + m[2] ** 2) / L
    expect = 1.0 + 0.3 * np.exp(-0.5 * kk * kk * R * R) * np.cos(phase + 0.4)
    if m == (8, 0, 0):
        expect = 1.0 + 0.3 * np.exp(-0.5 * kk * kk * R * R) * np.cos(0.4) * np.cos(phase)
    b = O.smooth_and_floor(rho, L, R, floor=0.05)
    assert np.max(np.abs(b - expect)) < 1e-13


def test_smoothing_floor_and_mean(O):
    """Without smoothing (R = 0) a two-valued field {0.01, 1.99} (mean 1)
    becomes {0.05, 1.99} / 1.02 exactly: the floor, then the mean restored."""
    N = 8
    rho = np.where(np.arange(N ** 3).reshape(N, N, N) % 2 == 0, 0.01, 1.99)
    b = O.smooth_and_floor(rho, 10.0, 0.0, floor=0.05)
    assert np.allclose(b, np.where(rho < 1, 0.05, 1.99) / 1.02, rtol=0, atol=1e-15)
    assert b.mean() == pytest.approx(1.0, abs=1e-15)


# --------------------------------------------------------------- adjoint
def test_jacobian_matches_finite_differences(O):
    N, h = 8, 1.0
    t = synth.smooth_field(N, 9, 0.4, kmax=2)
    v = np.random.default_rng(1).standard_normal((N,) * 3)
    eps = 1e-6
    fd = (O.det_grid(t + eps * v, h) - O.det_grid(t - eps * v, h)) / (2 * eps)
    assert np.allclose(O.jacobian_apply(t, v, h), fd, atol=1e-7)
    Jm = O.jacobian_matrix(t, h)
    assert np.allclose(Jm @ v.ravel(), fd.ravel(), atol=1e-7)


def test_adjoint_matches_finite_differences(O):
    """Gradient of loss = <w, theta(b)> against central differences of the
    oracle's own forward solve along random directions."""
    N, L = 8, 16.0
    h = L / N
    b = 1.0 + synth.smooth_field(N, 12, 0.5, kmax=2)
    t, _ = O.solve(b, L, tol=1e-14, max_cycles=80)
    w = np.random.default_rng(2).standard_normal((N,) * 3)
    g = O.adjoint(t, w, h)
    assert abs(g.sum()) < 1e-10 * np.abs(g).sum()
    rng = np.random.default_rng(3)
    for _ in range(3):
        d = rng.standard_normal((N,) * 3)
        eps = 1e-5
        tp, _ = O.solve(b + eps * d, L, theta0=t, tol=1e-14, max_cycles=80)
        tm, _ = O.solve(b - eps * d, L, theta0=t, tol=1e-14, max_cycles=80)
        fd = (np.sum(w * tp) - np.sum(w * tm)) / (2 * eps)
        assert np.sum(g * d) == pytest.approx(fd, rel=1e-6)


# --------------------------------------------------------------- cubic test
def test_cubic_test_interior(O):
    """Sec. III.A cubic test, scaled: 32^3 particles filling a cube of side
    2.5 at the centre of a 32^3 box (the paper's 10/128 ratio), CIC, floor.
    Inside the cube the map is a uniform scaling: Hbar = 0 and lap(theta) =
    3 (b_in^(1/3) - 1), the paper's 3 (L/l - 1) with the floor's mass taken
    out of b_in."""
    N, L, l = 32, 32.0, 2.5
    b = O.smooth_and_floor(O.cic_deposit(synth.cube_positions(N, L, l), N, L), L, 0.0)
    t, info = O.solve(b, L, tol=1e-3, max_cycles=80)
    assert info["status"] == 0
    c = N // 2
    H = [np.roll(t, -1, a) + np.roll(t, 1, a) - 2 * t for a in range(3)]   # h = 1
    lap = sum(H)[c - 1:c + 1, c - 1:c + 1, c - 1:c + 1]
    expect = 3.0 * (b[c, c, c] ** (1.0 / 3.0) - 1.0)
    assert np.all(np.abs(lap / expect - 1.0) < 1e-3)
    for a in range(3):
        hbar = H[a][c - 1:c + 1, c - 1:c + 1, c - 1:c + 1] - lap / 3.0
        assert np.max(np.abs(hbar)) < 1e-3 * expect


# --------------------------------------------------------------- Gaussianisation
def test_gaussianise_ranks_by_brute_force(O):
    """Ranks against the counting definition #(v_j < v_i) + #(j < i, v_j == v_i),
    with ties, both zero signs and negative values."""
    rng = np.random.default_rng(41)
    v = np.round(rng.standard_normal(300) * 3) / 2          # many ties
    v[:4] = [0.0, -0.0, 0.0, -0.0]
    _, rank = O.gaussianise(v)
    for i in range(v.size):
        assert rank[i] == np.sum(v < v[i]) + np.sum(v[:i] == v[i])


def test_gaussianise_properties(O):
    """The output keeps the input's order and mean, has the Gaussian
    quantiles as its values, is invariant (after standardising) under a
    monotonic map of the input, and leaves permuted Gaussian quantiles
    unchanged up to their own mean and std."""
    from scipy.special import ndtri
    rng = np.random.default_rng(42)
    v = rng.gamma(2.0, 1.0, (12, 12, 12)) - 2.0             # skewed
    g, rank = O.gaussianise(v)
    order = np.argsort(v, axis=None, kind="stable")
    assert np.all(np.diff(g.ravel()[order]) > 0)
    assert g.mean() == pytest.approx(v.mean(), abs=1e-12)
    q = ndtri((np.arange(v.size) + 0.5) / v.size)
    assert np.allclose(np.sort(g.ravel()), v.mean() + v.std() * q, atol=1e-12)
    g2, _ = O.gaussianise(np.exp(v))
    z = lambda a: (a - a.mean()) / a.std()
    assert np.allclose(z(g2), z(g), atol=1e-12)
    perm = rng.permutation(v.size)
    w = q[perm]
    gw, _ = O.gaussianise(w)
    assert np.allclose(gw, w.mean() + w.std() * w, atol=1e-12)


# --------------------------------------------------------------- mutations
MUTATIONS = {
    "edge-sign": ("- t[at(N, i - 1, j + 1, k)] - t[at(N, i + 1, j - 1, k)]) / q4;",
                  "+ t[at(N, i - 1, j + 1, k)] - t[at(N, i + 1, j - 1, k)]) / q4;"),
    "det-drop-yz": ("return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])",
                    "return A[0][0] * (A[1][1] * A[2][2])"),
    "printed-root-branch": ("return 2.0 * sqrt(-p / 3.0) * cos(sigma / 3.0);",
                            "return 2.0 * sqrt(-p / 3.0) * cos((sigma + 2.0 * M_PI) / 3.0);"),
    "prolong-weight": ("double w = (a ? 0.25 : 0.75) * (b ? 0.25 : 0.75)",
                       "double w = (a ? 0.5 : 0.5) * (b ? 0.25 : 0.75)"),
    "restrict-index": ("acc += f[at(Nf, 2 * I + a, 2 * J + b, 2 * K + cc)];",
                       "acc += f[at(Nf, 2 * I + a, 2 * J + b, 2 * K)];"),
    "no-compat": ("        c -= m;\n        double mt", "        double mt"),
    "tsc-side": ("w[a][0] = 0.5 * (0.5 - d[a]) * (0.5 - d[a]);",
                 "w[a][0] = 0.5 * (0.5 + d[a]) * (0.5 + d[a]);"),
    "ngp-cell": ("rho[at(N, i[0], i[1], i[2])] += mass;",
                 "rho[at(N, i[0], i[1], i[2] + 1)] += mass;"),
    "displace-q-sign": ("double qq = fmod(x[d] + g[d], L);",
                        "double qq = fmod(x[d] - g[d], L);"),
    "displace-den-unweighted": ("wb[id] = b[id];", "wb[id] = 1.0;"),
    "displace-v-sign": ("double v = 3.0 - inv_tr;", "double v = inv_tr - 3.0;"),
    "smooth-window-exponent": ("oracle.py", "np.exp(-0.5 * k2 * R * R)", "np.exp(-k2 * R * R)"),
    "smooth-no-renorm": ("oracle.py", "    b = np.maximum(r, floor)\n    return b / b.mean()",
                         "    b = np.maximum(r, floor)\n    return b"),
    "cic-offset": ("double u = x * ((double)N / L) - 0.5;", "double u = x * ((double)N / L);"),
    "cic-weight-swap": ("double w = (a ? f[0] : 1.0 - f[0]) * (b ? f[1] : 1.0 - f[1])\n"
                        "                             * (cc ? f[2] : 1.0 - f[2]);\n"
                        "                    rho[at(N, i0[0] + a, i0[1] + b, i0[2] + cc)] += mass * w;",
                        "double w = (a ? 1.0 - f[0] : f[0]) * (b ? f[1] : 1.0 - f[1])\n"
                        "                             * (cc ? f[2] : 1.0 - f[2]);\n"
                        "                    rho[at(N, i0[0] + a, i0[1] + b, i0[2] + cc)] += mass * w;"),
    "coarse-rhs-sign": ("Hh->g[l + 1][x] = dH[x] + sc * rr[x];", "Hh->g[l + 1][x] = dH[x] - sc * rr[x];"),
    "jacobian-row-mixed-once": ("double wxy = 2.0 * cxy / (4.0 * h2);", "double wxy = cxy / (4.0 * h2);"),
    "jacobian-apply-mixed-once": ("+ 2.0 * (cof[3 * n + id] * D[0][1]", "+ (cof[3 * n + id] * D[0][1]"),
    "adjoint-no-transpose": ("oracle.py", "AT = A.T.tocsc()", "AT = A.tocsc()"),
    "gauss-no-mean": ("oracle.py", "g = v.mean() + v.std() * ndtri(", "g = v.std() * ndtri("),
    "traceless-half": ("Hb[a][b] = H[a][b] - (a == b ? tr / 3.0 : 0.0);",
                       "Hb[a][b] = H[a][b] - (a == b ? tr / 2.0 : 0.0);"),
    "eps-no-compat": ("or_cell_cubic(t, N, h, i, j, k, g[at(N, i, j, k)] + c, &s, &p, &q);\n                double L",
                      "or_cell_cubic(t, N, h, i, j, k, g[at(N, i, j, k)], &s, &p, &q);\n                double L"),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutations_are_caught(O, name, tmp_path):
    """Plant a plausible mistake in a copy of the oracle: a pin must fail."""
    import importlib.util
    import os
    import shutil
    src_dir = os.path.dirname(O.__file__)
    shutil.copy(os.path.join(src_dir, "recon_oracle.c"), tmp_path / "recon_oracle.c")
    shutil.copy(os.path.join(src_dir, "oracle.py"), tmp_path / "oracle.py")
    entry = MUTATIONS[name]
    fname, old, new = entry if len(entry) == 3 else ("recon_oracle.c", *entry)
    code = (tmp_path / fname).read_text()
    assert code.count(old) == 1, name
    (tmp_path / fname).write_text(code.replace(old, new))
    spec = importlib.util.spec_from_file_location(f"mut_{name.replace('-', '_')}",
                                                  tmp_path / "oracle.py")
    M = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(M)
    pins = [
        lambda: test_plane_cubic_worked_values(M, 4.0, 7.0),
        lambda: test_cubic_is_27_det(M),
        lambda: test_appendix_A2_fixed_equals_oracle_q(M),
        lambda: test_diagonal_plane_wave(M, (0, 1, 2)),
        lambda: test_plane_symmetric_closed_form(M, 0),
        lambda: test_separable_potential(M),
        lambda: test_restriction_is_eight_son_mean(M),
        lambda: test_prolongation_reproduces_linear_fields(M),
        lambda: test_assignment_is_the_cardinal_bspline(M, "ngp", 0),
        lambda: test_assignment_is_the_cardinal_bspline(M, "tsc", 2),
        lambda: test_displace_recovers_plane_zeldovich(M, 0.5),
        lambda: test_paper_eps_plane_closed_form(M),
        lambda: test_smoothing_window_on_single_modes(M, (1, 2, 3)),
        lambda: test_smoothing_floor_and_mean(M),
        lambda: test_cic_textbook_definition(M),
        lambda: test_jacobian_matches_finite_differences(M),
        lambda: test_adjoint_matches_finite_differences(M),
        lambda: test_gaussianise_properties(M),
    ]
    failed = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed >= 1, f"mutation {name} passed every pin"


def test_defect_scale_safeguard(O):
    """Scaled-defect factor: 1 when the coarse right side stays positive,
    floor * det / (-R d) where it would not, 0 (skip) when det <= 0."""
    d = np.array([1.0, 2.0, 0.5])
    assert O.defect_scale(d, np.array([0.3, -0.5, 0.1]), 0.5) == 1.0
    assert O.defect_scale(d, np.array([0.3, -4.0, 0.1]), 0.5) == pytest.approx(0.25)
    assert O.defect_scale(np.array([-0.1, 1.0]), np.array([-0.2, 0.0]), 0.5) == 0.0
    assert O.defect_scale(d, -10 * d, 0.0) == 1.0
