"""Identities behind the FP32 smoothers' rearranged arithmetic (no GPU).

The paired-FP32 updates of the fused sweep evaluate the cell cubic of
Sec. II (eqs. final_PDE2, update) and the linear smoother of the defect
correction in a rearranged but algebraically equal form, and keep a Newton
step by a cancellation-free test.  These tests prove the rearrangements
symbolically and check the test's decision in exact rational arithmetic.
"""
from fractions import Fraction

import numpy as np
import pytest

sp = pytest.importorskip("sympy")


def test_newton_value_identity():
    """f(s - u) = u^2 (3 s - u) for the Newton quotient u = f(s) / f'(s) of
    f = s^3 + p s + q: the new |f| needs no recomputation of f."""
    s, p, q = sp.symbols("s p q")
    f = s**3 + p * s + q
    u = f / sp.diff(f, s)
    assert sp.simplify(f.subs(s, s - u) - u**2 * (3 * s - u)) == 0


def test_newton_keep_decision_exact():
    """|u (3 s - u)| <= f'(s) decides exactly as |f(s - u)| <= |f(s)| (exact
    rationals; f' > 0 and s > 0, the region where the step is tried)."""
    rng = np.random.default_rng(5)
    n = 0
    for _ in range(3000):
        p = Fraction(-abs(rng.standard_normal()) * rng.choice([0.1, 1.0, 30.0]))
        q = Fraction(rng.standard_normal() * rng.choice([1.0, 30.0]))
        s = Fraction(rng.uniform(0.05, 8.0))
        fp = 3 * s * s + p
        if fp <= 0:
            continue
        f = s**3 + p * s + q
        u = f / fp
        sn = s - u
        old = abs(sn**3 + p * sn + q) <= abs(f)
        new = abs(u * (3 * s - u)) <= fp
        assert old == new
        n += 1
    assert n > 1000


def test_paired_fas_coefficients_equal_scalar_form():
    """Hbar_aa = S_a ih2 - (S_x+S_y+S_z) ih2/3 equals (2 S_a - S_b - S_c) ih2/3,
    and s = 3 + (S - 6 c) ih2 is the same in both forms."""
    X, Y, Z, ih2 = sp.symbols("X Y Z ih2")
    Sg = X + Y + Z
    for a, b, c in ((X, Y, Z), (Y, Z, X), (Z, X, Y)):
        assert sp.expand(a * ih2 - Sg * ih2 / 3 - (2 * a - b - c) * ih2 / 3) == 0


def test_paired_theta_update_equals_eq_update():
    """theta_c - (h^2/6)(s_new - s) with s_new = s - u is theta_c + (h^2/6) u."""
    th, h, s, u = sp.symbols("theta h s u")
    assert sp.expand(th - h**2 / 6 * ((s - u) - s) - (th + h**2 / 6 * u)) == 0


def test_paired_linear_update_equals_gauss_seidel():
    """e_c + (J'e/2 - h^2 f/2) / tr(adj) equals e_c + (f - J e) / J_cc with
    J e = sum_ab adj_ab D_ab e (1/h^2 stencils), J'e = h^2 J e and
    J_cc = -2 tr(adj) / h^2."""
    ec, f, h, T, Jp = sp.symbols("e_c f h T Jp", nonzero=True)
    Je = Jp / h**2
    Jcc = -2 * T / h**2
    lhs = ec + (Jp / 2 - h**2 * f / 2) / T
    rhs = ec + (f - Je) / Jcc
    assert sp.simplify(lhs - rhs) == 0


def test_paired_linear_edge_scaling():
    """The off-diagonal terms: 2 adj_ab (E_ab / (4 h^2)) h^2 = adj_ab E_ab / 2
    for the unscaled 4-point edge combination E_ab."""
    a, E, h = sp.symbols("a E h", nonzero=True)
    assert sp.simplify(2 * a * (E / (4 * h**2)) * h**2 - a * E / 2) == 0
